// k_dd.cu -- FFT and per-frequency product kernels instantiated for dd.
#include "launchers.cuh"
MRC_DEFINE_PREC(dd, dd)
