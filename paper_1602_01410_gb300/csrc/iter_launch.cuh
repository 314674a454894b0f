// Launch wrappers for the iteration kernels: dispatch on CTA size (256 or
// 512 threads) and channel count (1, or 3 for vectorial TV).
#pragma once

#include "iter_kernels.cuh"

namespace dcv {

template <typename T, int NT, int C>
static cudaError_t row_launch_nt(const RowArgs<T> &a, int grid, size_t smem, cudaStream_t s) {
  row_pass_kernel<T, NT, C><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

// 512-thread CTAs exist for FP32 only (FP64 registers would spill).
template <typename T> constexpr int kMaxNt = sizeof(T) == 4 ? 512 : 256;

template <typename T>
cudaError_t launch_row(const RowArgs<T> &a, int grid, int nt, int channels, size_t smem, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  if (nt == 512 && kMaxNt<T> == 512)
    return channels == 3 ? row_launch_nt<T, kMaxNt<T>, 3>(a, grid, smem, s) : row_launch_nt<T, kMaxNt<T>, 1>(a, grid, smem, s);
  if (nt != 256) return cudaErrorInvalidValue;
  return channels == 3 ? row_launch_nt<T, 256, 3>(a, grid, smem, s) : row_launch_nt<T, 256, 1>(a, grid, smem, s);
}

template <typename T>
cudaError_t launch_col(const ColArgs<T> &a, int grid, int nt, size_t smem, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  if (nt == 512 && kMaxNt<T> == 512) col_pass_kernel<T, kMaxNt<T>><<<grid, kMaxNt<T>, smem, s>>>(a);
  else if (nt == 256) col_pass_kernel<T, 256><<<grid, 256, smem, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// Opt in to the dynamic shared memory the plan needs (above 48 KB).
template <typename T>
cudaError_t prepare_kernels(int nt, int channels, size_t row_smem, size_t col_smem) {
  cudaError_t e;
  const int rs = (int)row_smem, cs = (int)col_smem;
  if (nt == 512 && kMaxNt<T> == 512) {
    constexpr int NT = kMaxNt<T>;
    e = channels == 3 ? cudaFuncSetAttribute(row_pass_kernel<T, NT, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)
                      : cudaFuncSetAttribute(row_pass_kernel<T, NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(col_pass_kernel<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs);
  }
  if (nt != 256) return cudaErrorInvalidValue;
  e = channels == 3 ? cudaFuncSetAttribute(row_pass_kernel<T, 256, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs)
                    : cudaFuncSetAttribute(row_pass_kernel<T, 256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(col_pass_kernel<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs);
}

}  // namespace dcv
