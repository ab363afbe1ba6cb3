// k_f64_fft_hi.cu -- FFT pass kernels for double, radices 2^7 .. 2^10.
#include "kernels.cuh"
void mrc_fft_fill_f64_hi(FftEntry (*t)[11], FftSegEntry *ts) { fft_fill_shifted<double, 7>(t, ts, std::make_integer_sequence<int, 4>{}); }
