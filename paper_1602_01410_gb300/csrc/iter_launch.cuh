// Launch wrappers for the iteration kernels: resolve the kernel of a
// LaunchCfg (generic Stockham passes by CTA size and channel count, or the
// register-FFT passes by threads per transform, radix and channel count).
#pragma once

#include "iter_kernels.cuh"

namespace dcv {

// 512-thread generic CTAs exist for FP32 only (FP64 registers would spill).
template <typename T> constexpr int kMaxNt = sizeof(T) == 4 ? 512 : 256;

// Register-FFT passes of lengths R * 32 * TT (TT = tt): the kernels live in
// one translation unit per (type, R) (p2_tables.cuh), which compile in
// parallel.  half 0: inverse half, 1: forward half (stage 0 reads through
// L1, 1 stages its rows (one channel), 2 adds penalty adaptation), 2: the y~
// spectrum of an inner pass, 3: the fused row pass of a plain iteration.
template <typename T, int R> const void *p2_row_kernel(int C, int tt, int v, int half, int stage);
template <typename T, int R> const void *p2_col_kernel(int tt, int v, int ext);

template <typename T>
static const void *p2_row_ptr(int C, int tt, int r, int v, int half, int stage) {
  switch (r) {
    case 1: return p2_row_kernel<T, 1>(C, tt, v, half, stage);
    case 3: return p2_row_kernel<T, 3>(C, tt, v, half, stage);
    case 5: return p2_row_kernel<T, 5>(C, tt, v, half, stage);
  }
  return nullptr;
}

template <typename T>
static const void *row_ptr(const LaunchCfg &c, int half = 0) {
  if (c.kind == KIND_P2) return p2_row_ptr<T>(c.channels, c.tt, c.r, c.v ? c.v : 32, half, c.stage);
  if (c.nt == 512 && kMaxNt<T> == 512)
    return c.channels == 3 ? (const void *)row_pass_kernel<T, kMaxNt<T>, 3> : (const void *)row_pass_kernel<T, kMaxNt<T>, 1>;
  if (c.nt == 256)
    return c.channels == 3 ? (const void *)row_pass_kernel<T, 256, 3> : (const void *)row_pass_kernel<T, 256, 1>;
  return nullptr;
}

template <typename T>
static const void *col_ptr(const LaunchCfg &c) {
  if (c.kind == KIND_P2) {
    switch (c.r) {
      case 1: return p2_col_kernel<T, 1>(c.tt, c.v ? c.v : 32, c.stage);
      case 3: return p2_col_kernel<T, 3>(c.tt, c.v ? c.v : 32, c.stage);
      case 5: return p2_col_kernel<T, 5>(c.tt, c.v ? c.v : 32, c.stage);
    }
    return nullptr;
  }
  if (c.nt == 512 && kMaxNt<T> == 512) return (const void *)col_pass_kernel<T, kMaxNt<T>>;
  if (c.nt == 256) return (const void *)col_pass_kernel<T, 256>;
  return nullptr;
}

// The iteration kernels use programmatic dependent launch: a kernel may
// start while its predecessor finishes, and waits in griddep_wait() before
// it touches the state.
template <typename A>
static cudaError_t launch_ptr(const void *fn, const A &a, const LaunchCfg &c, cudaStream_t s) {
  if (!fn) return cudaErrorInvalidValue;
  if (c.grid <= 0) return cudaSuccess;
  void *args[] = {const_cast<A *>(&a)};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(c.grid);
  lc.blockDim = dim3(c.nt);
  lc.dynamicSmemBytes = c.smem;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  return cudaLaunchKernelExC(&lc, fn, args);
}

// The configuration of one half of a register-FFT row pass (its own shared
// memory size; the fused pass uses the inverse half's).
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

// One half of a power-of-two row pass (0: inverse, 1: forward, 2: y~
// spectrum, 3: the fused pass).  Kernels are
// launched from the translation unit that opted them in to their shared
// memory (each unit instantiates its own copy of a kernel template).
template <typename T>
cudaError_t launch_row_half(const RowArgs<T> &a, const LaunchCfg &c, int half, cudaStream_t s) {
  return launch_ptr(row_ptr<T>(c, half), a, row_half_cfg(c, half), s);
}

// Opt in to the dynamic shared memory a class needs (above 48 KB).  The
// shared-memory carve-out is left to the driver, which sizes it for the
// occupancy the other limits allow and leaves the rest to L1 (the forward
// row half reads its neighbours' rows through L1).
static inline cudaError_t opt_in_smem(const void *fn, size_t smem) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
cudaError_t prepare_row(const LaunchCfg &c) {
  for (int half = 0; half < (c.kind == KIND_P2 ? 4 : 1); ++half) {
    const void *fn = row_ptr<T>(c, half);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = opt_in_smem(fn, row_half_cfg(c, half).smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t prepare_col(const LaunchCfg &c) {
  for (int ext = 0; ext < (c.kind == KIND_P2 ? 2 : 1); ++ext) {
    LaunchCfg e = c;
    e.stage = ext;
    const void *fn = col_ptr<T>(e);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t r = opt_in_smem(fn, c.smem);
    if (r != cudaSuccess) return r;
  }
  return cudaSuccess;
}

}  // namespace dcv
