// FP32 register-FFT passes of lengths 5*2^k.
#include "p2_tables.cuh"

DCV_P2_INSTANTIATE(float, 5)
