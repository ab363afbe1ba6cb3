// k_f32.cu -- FFT and per-frequency product kernels instantiated for float.
#include "launchers.cuh"
MRC_DEFINE_PREC(float, f32)
