// k_f64_fft_lo.cu -- FFT pass kernels for double, radices 2^0 .. 2^6.
#include "kernels.cuh"
void mrc_fft_fill_f64_lo(FftEntry (*t)[11], FftSegEntry *ts) { fft_fill_shifted<double, 0>(t, ts, std::make_integer_sequence<int, 7>{}); }
