// Kernel tables of the register-FFT passes for one (type, radix R): each
// p2_*.cu translation unit includes this file and instantiates one pair, so
// that every kernel instance exists in exactly one unit (the shared-memory
// opt-in and the launch go through the same function pointer).
#pragma once

#include "iter_fused.cuh"
#include "iter_launch.cuh"
#include "iter_p2.cuh"

namespace dcv {

template <typename T, int TT, int C, int R, int V>
static const void *p2_row_one(int half, int stage) {
  if (!half) return (const void *)row_inv_p2_kernel<T, TT, C, R, V>;
  if (half == 2) return (const void *)row_yspec_p2_kernel<T, TT, C, R, V>;
  if (half == 3) return (const void *)row_fused_p2_kernel<T, TT, C, R, V>;
  if (stage == 2) return (const void *)row_fwd_p2_kernel<T, TT, C, R, true, V>;  // penalty adaptation
  if constexpr (C == 1)
    if (stage == 1) return (const void *)row_fwd_p2_staged_kernel<T, TT, C, R, V>;
  return (const void *)row_fwd_p2_kernel<T, TT, C, R, false, V>;
}

template <typename T, int C, int R>
static const void *p2_row_tt(int tt, int v, int half, int stage) {
  if constexpr (R == 1) {
    if (v == 16) {
      switch (tt) {
        case 4: return p2_row_one<T, 4, C, R, 16>(half, stage);
        case 8: return p2_row_one<T, 8, C, R, 16>(half, stage);
        case 16: return p2_row_one<T, 16, C, R, 16>(half, stage);
        case 32: return p2_row_one<T, 32, C, R, 16>(half, stage);
        case 64: return p2_row_one<T, 64, C, R, 16>(half, stage);
      }
      return nullptr;
    }
    switch (tt) {
      case 2: return p2_row_one<T, 2, C, R, 32>(half, stage);
      case 4: return p2_row_one<T, 4, C, R, 32>(half, stage);
      case 8: return p2_row_one<T, 8, C, R, 32>(half, stage);
      case 16: return p2_row_one<T, 16, C, R, 32>(half, stage);
      case 32: return p2_row_one<T, 32, C, R, 32>(half, stage);
    }
  } else {
    if (v == 16) {
      switch (tt) {
        case 8: return p2_row_one<T, 8, C, R, 16>(half, stage);
        case 16: return p2_row_one<T, 16, C, R, 16>(half, stage);
        case 32: return p2_row_one<T, 32, C, R, 16>(half, stage);
      }
      return nullptr;
    }
    switch (tt) {
      case 4: return p2_row_one<T, 4, C, R, 32>(half, stage);
      case 8: return p2_row_one<T, 8, C, R, 32>(half, stage);
      case 16: return p2_row_one<T, 16, C, R, 32>(half, stage);
    }
  }
  return nullptr;
}

template <typename T, int R> const void *p2_row_kernel(int C, int tt, int v, int half, int stage) {
  return C == 3 ? p2_row_tt<T, 3, R>(tt, v, half, stage) : p2_row_tt<T, 1, R>(tt, v, half, stage);
}

template <typename T, int R, bool EXT> static const void *p2_col_tt(int tt, int v) {
  if constexpr (R == 1) {
    if (v == 16) {
      switch (tt) {
        case 4: return (const void *)col_pass_p2_kernel<T, 4, R, EXT, 16>;
        case 8: return (const void *)col_pass_p2_kernel<T, 8, R, EXT, 16>;
        case 16: return (const void *)col_pass_p2_kernel<T, 16, R, EXT, 16>;
        case 32: return (const void *)col_pass_p2_kernel<T, 32, R, EXT, 16>;
        case 64: return (const void *)col_pass_p2_kernel<T, 64, R, EXT, 16>;
      }
      return nullptr;
    }
    switch (tt) {
      case 2: return (const void *)col_pass_p2_kernel<T, 2, R, EXT, 32>;
      case 4: return (const void *)col_pass_p2_kernel<T, 4, R, EXT, 32>;
      case 8: return (const void *)col_pass_p2_kernel<T, 8, R, EXT, 32>;
      case 16: return (const void *)col_pass_p2_kernel<T, 16, R, EXT, 32>;
      case 32: return (const void *)col_pass_p2_kernel<T, 32, R, EXT, 32>;
    }
  } else {
    if (v == 16) {
      switch (tt) {
        case 8: return (const void *)col_pass_p2_kernel<T, 8, R, EXT, 16>;
        case 16: return (const void *)col_pass_p2_kernel<T, 16, R, EXT, 16>;
        case 32: return (const void *)col_pass_p2_kernel<T, 32, R, EXT, 16>;
      }
      return nullptr;
    }
    switch (tt) {
      case 4: return (const void *)col_pass_p2_kernel<T, 4, R, EXT, 32>;
      case 8: return (const void *)col_pass_p2_kernel<T, 8, R, EXT, 32>;
      case 16: return (const void *)col_pass_p2_kernel<T, 16, R, EXT, 32>;
    }
  }
  return nullptr;
}

// ext: the variant with the Tikhonov step and the per-image penalty.
template <typename T, int R> const void *p2_col_kernel(int tt, int v, int ext) {
  return ext ? p2_col_tt<T, R, true>(tt, v) : p2_col_tt<T, R, false>(tt, v);
}

}  // namespace dcv

#define DCV_P2_INSTANTIATE(T, R)                                                   \
  namespace dcv {                                                                  \
  template const void *p2_row_kernel<T, R>(int C, int tt, int v, int half, int stage); \
  template const void *p2_col_kernel<T, R>(int tt, int v, int ext);                \
  }
