// k_dd_fft_lo.cu -- FFT pass kernels for dd, radices 2^0 .. 2^6.
#include "kernels.cuh"
void mrc_fft_fill_dd_lo(FftEntry (*t)[11], FftSegEntry *ts) { fft_fill_shifted<dd, 0>(t, ts, std::make_integer_sequence<int, 7>{}); }
