// Kernel tables of the register-FFT passes for one (type, radix R): each
// p2_*.cu translation unit includes this file and instantiates one pair, so
// that every kernel instance exists in exactly one unit (the shared-memory
// opt-in and the launch go through the same function pointer).
#pragma once

#include "iter_launch.cuh"
#include "iter_p2.cuh"

namespace dcv {

template <typename T, int TT, int C, int R>
static const void *p2_row_one(int half, int stage) {
  if (!half) return (const void *)row_inv_p2_kernel<T, TT, C, R>;
  if (half == 2) return (const void *)row_yspec_p2_kernel<T, TT, C, R>;
  if (stage == 2) return (const void *)row_fwd_p2_kernel<T, TT, C, R, true>;  // penalty adaptation
  if constexpr (C == 1)
    if (stage == 1) return (const void *)row_fwd_p2_staged_kernel<T, TT, C, R>;
  return (const void *)row_fwd_p2_kernel<T, TT, C, R, false>;
}

template <typename T, int C, int R>
static const void *p2_row_tt(int tt, int half, int stage) {
  if constexpr (R == 1) {
    switch (tt) {
      case 2: return p2_row_one<T, 2, C, R>(half, stage);
      case 4: return p2_row_one<T, 4, C, R>(half, stage);
      case 8: return p2_row_one<T, 8, C, R>(half, stage);
      case 16: return p2_row_one<T, 16, C, R>(half, stage);
      case 32: return p2_row_one<T, 32, C, R>(half, stage);
    }
  } else {
    switch (tt) {
      case 4: return p2_row_one<T, 4, C, R>(half, stage);
      case 8: return p2_row_one<T, 8, C, R>(half, stage);
      case 16: return p2_row_one<T, 16, C, R>(half, stage);
    }
  }
  return nullptr;
}

template <typename T, int R> const void *p2_row_kernel(int C, int tt, int half, int stage) {
  return C == 3 ? p2_row_tt<T, 3, R>(tt, half, stage) : p2_row_tt<T, 1, R>(tt, half, stage);
}

template <typename T, int R, bool EXT> static const void *p2_col_tt(int tt) {
  if constexpr (R == 1) {
    switch (tt) {
      case 2: return (const void *)col_pass_p2_kernel<T, 2, R, EXT>;
      case 4: return (const void *)col_pass_p2_kernel<T, 4, R, EXT>;
      case 8: return (const void *)col_pass_p2_kernel<T, 8, R, EXT>;
      case 16: return (const void *)col_pass_p2_kernel<T, 16, R, EXT>;
      case 32: return (const void *)col_pass_p2_kernel<T, 32, R, EXT>;
    }
  } else {
    switch (tt) {
      case 4: return (const void *)col_pass_p2_kernel<T, 4, R, EXT>;
      case 8: return (const void *)col_pass_p2_kernel<T, 8, R, EXT>;
      case 16: return (const void *)col_pass_p2_kernel<T, 16, R, EXT>;
    }
  }
  return nullptr;
}

// ext: the variant with the Tikhonov step and the per-image penalty.
template <typename T, int R> const void *p2_col_kernel(int tt, int ext) {
  return ext ? p2_col_tt<T, R, true>(tt) : p2_col_tt<T, R, false>(tt);
}

}  // namespace dcv

#define DCV_P2_INSTANTIATE(T, R)                                                   \
  namespace dcv {                                                                  \
  template const void *p2_row_kernel<T, R>(int C, int tt, int half, int stage);    \
  template const void *p2_col_kernel<T, R>(int tt, int ext);                       \
  }
