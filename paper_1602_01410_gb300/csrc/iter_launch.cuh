// Launch wrappers for the iteration kernels: resolve the kernel of a
// LaunchCfg (generic Stockham passes by CTA size and channel count, or the
// power-of-two passes by threads per transform and channel count).
#pragma once

#include "iter_kernels.cuh"
#include "iter_p2.cuh"

namespace dcv {

// 512-thread generic CTAs exist for FP32 only (FP64 registers would spill).
template <typename T> constexpr int kMaxNt = sizeof(T) == 4 ? 512 : 256;

// Power-of-two and R * 2^k row passes: half 0 = inverse (R1), half 1 = forward (R2).
// The staged forward half exists for one channel only.
template <typename T, int TT, int C, int R>
static const void *row_p2_one(int half, int stage) {
  if (!half) return (const void *)row_inv_p2_kernel<T, TT, C, R>;
  if constexpr (C == 1)
    if (stage) return (const void *)row_fwd_p2_staged_kernel<T, TT, C, R>;
  return (const void *)row_fwd_p2_kernel<T, TT, C, R>;
}

template <typename T, int C>
static const void *row_p2_ptr(int tt, int r, int half, int stage) {
  if (r == 1) {
    switch (tt) {
      case 2: return row_p2_one<T, 2, C, 1>(half, stage);
      case 4: return row_p2_one<T, 4, C, 1>(half, stage);
      case 8: return row_p2_one<T, 8, C, 1>(half, stage);
      case 16: return row_p2_one<T, 16, C, 1>(half, stage);
      case 32: return row_p2_one<T, 32, C, 1>(half, stage);
    }
  } else if (r == 3) {
    switch (tt) {
      case 4: return row_p2_one<T, 4, C, 3>(half, stage);
      case 8: return row_p2_one<T, 8, C, 3>(half, stage);
      case 16: return row_p2_one<T, 16, C, 3>(half, stage);
    }
  } else if (r == 5) {
    switch (tt) {
      case 4: return row_p2_one<T, 4, C, 5>(half, stage);
      case 8: return row_p2_one<T, 8, C, 5>(half, stage);
      case 16: return row_p2_one<T, 16, C, 5>(half, stage);
    }
  }
  return nullptr;
}

template <typename T>
static const void *row_ptr(const LaunchCfg &c, int half = 0) {
  if (c.kind == KIND_P2)
    return c.channels == 3 ? row_p2_ptr<T, 3>(c.tt, c.r, half, c.stage) : row_p2_ptr<T, 1>(c.tt, c.r, half, c.stage);
  if (c.nt == 512 && kMaxNt<T> == 512)
    return c.channels == 3 ? (const void *)row_pass_kernel<T, kMaxNt<T>, 3> : (const void *)row_pass_kernel<T, kMaxNt<T>, 1>;
  if (c.nt == 256)
    return c.channels == 3 ? (const void *)row_pass_kernel<T, 256, 3> : (const void *)row_pass_kernel<T, 256, 1>;
  return nullptr;
}

template <typename T>
static const void *col_ptr(const LaunchCfg &c) {
  if (c.kind == KIND_P2) {
    if (c.r == 1) {
      switch (c.tt) {
        case 2: return (const void *)col_pass_p2_kernel<T, 2, 1>;
        case 4: return (const void *)col_pass_p2_kernel<T, 4, 1>;
        case 8: return (const void *)col_pass_p2_kernel<T, 8, 1>;
        case 16: return (const void *)col_pass_p2_kernel<T, 16, 1>;
        case 32: return (const void *)col_pass_p2_kernel<T, 32, 1>;
      }
    } else if (c.r == 3) {
      switch (c.tt) {
        case 4: return (const void *)col_pass_p2_kernel<T, 4, 3>;
        case 8: return (const void *)col_pass_p2_kernel<T, 8, 3>;
        case 16: return (const void *)col_pass_p2_kernel<T, 16, 3>;
      }
    } else if (c.r == 5) {
      switch (c.tt) {
        case 4: return (const void *)col_pass_p2_kernel<T, 4, 5>;
        case 8: return (const void *)col_pass_p2_kernel<T, 8, 5>;
        case 16: return (const void *)col_pass_p2_kernel<T, 16, 5>;
      }
    }
    return nullptr;
  }
  if (c.nt == 512 && kMaxNt<T> == 512) return (const void *)col_pass_kernel<T, kMaxNt<T>>;
  if (c.nt == 256) return (const void *)col_pass_kernel<T, 256>;
  return nullptr;
}

template <typename A>
static cudaError_t launch_ptr(const void *fn, const A &a, const LaunchCfg &c, cudaStream_t s) {
  if (!fn) return cudaErrorInvalidValue;
  if (c.grid <= 0) return cudaSuccess;
  void *args[] = {const_cast<A *>(&a)};
  return cudaLaunchKernel(fn, dim3(c.grid), dim3(c.nt), args, c.smem, s);
}

// The configuration of one half of a register-FFT row pass (its own shared memory size).
static inline LaunchCfg row_half_cfg(const LaunchCfg &c, int half) {
  LaunchCfg h = c;
  if (c.kind == KIND_P2 && half == 1) h.smem = c.smem_fwd;
  return h;
}

template <typename T>
cudaError_t launch_row(const RowArgs<T> &a, const LaunchCfg &c, cudaStream_t s) {
  cudaError_t e = launch_ptr(row_ptr<T>(c, 0), a, c, s);
  if (e != cudaSuccess || c.kind != KIND_P2) return e;
  return launch_ptr(row_ptr<T>(c, 1), a, row_half_cfg(c, 1), s);
}

template <typename T>
cudaError_t launch_col(const ColArgs<T> &a, const LaunchCfg &c, cudaStream_t s) {
  return launch_ptr(col_ptr<T>(c), a, c, s);
}

// One half of a power-of-two row pass (0: inverse, 1: forward).  Kernels are
// launched from the translation unit that opted them in to their shared
// memory (each unit instantiates its own copy of a kernel template).
template <typename T>
cudaError_t launch_row_half(const RowArgs<T> &a, const LaunchCfg &c, int half, cudaStream_t s) {
  return launch_ptr(row_ptr<T>(c, half), a, row_half_cfg(c, half), s);
}

// Opt in to the dynamic shared memory a class needs (above 48 KB).
template <typename T>
cudaError_t prepare_row(const LaunchCfg &c) {
  for (int half = 0; half < (c.kind == KIND_P2 ? 2 : 1); ++half) {
    const void *fn = row_ptr<T>(c, half);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_half_cfg(c, half).smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t prepare_col(const LaunchCfg &c) {
  const void *fn = col_ptr<T>(c);
  if (!fn) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
}

}  // namespace dcv
