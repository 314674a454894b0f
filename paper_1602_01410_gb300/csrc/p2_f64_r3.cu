// FP64 register-FFT passes of lengths 3*2^k.
#include "p2_tables.cuh"

DCV_P2_INSTANTIATE(double, 3)
