// k_f64.cu -- FFT and per-frequency product kernels instantiated for double.
#include "launchers.cuh"
MRC_DEFINE_PREC(double, f64)
