// k_f32_fft_hi.cu -- FFT pass kernels for float, radices 2^7 .. 2^10.
#include "kernels.cuh"
void mrc_fft_fill_f32_hi(FftEntry (*t)[11], FftSegEntry *ts) { fft_fill_shifted<float, 7>(t, ts, std::make_integer_sequence<int, 4>{}); }
