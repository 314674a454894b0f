// Launchers of the reverse-pass kernels (FP32 and FP64).
#include "adjoint.cuh"

namespace dcv {

template <typename T, int C>
static const void *adj_ptr_c(int N, int v) {
  if (v == 16) {
    switch (N / 16) {
      case 4: return (const void *)row_adj_p2_kernel<T, 4, C, 1, 16>;
      case 8: return (const void *)row_adj_p2_kernel<T, 8, C, 1, 16>;
      case 16: return (const void *)row_adj_p2_kernel<T, 16, C, 1, 16>;
      case 32: return (const void *)row_adj_p2_kernel<T, 32, C, 1, 16>;
      case 64: return (const void *)row_adj_p2_kernel<T, 64, C, 1, 16>;
    }
    return nullptr;
  }
  switch (N / 32) {
    case 2: return (const void *)row_adj_p2_kernel<T, 2, C, 1, 32>;
    case 4: return (const void *)row_adj_p2_kernel<T, 4, C, 1, 32>;
    case 8: return (const void *)row_adj_p2_kernel<T, 8, C, 1, 32>;
    case 16: return (const void *)row_adj_p2_kernel<T, 16, C, 1, 32>;
    case 32: return (const void *)row_adj_p2_kernel<T, 32, C, 1, 32>;
  }
  return nullptr;
}

// Lengths 3 * 2^k and 5 * 2^k come from adjoint_r35.cu (16 values per thread).
template <typename T>
static const void *adj_ptr(int N, int v, int C) {
  if (N % 3 == 0 || N % 5 == 0) return adj_ptr_r35<T>(N, v, C);
  return C == 3 ? adj_ptr_c<T, 3>(N, v) : adj_ptr_c<T, 1>(N, v);
}

template <typename T>
cudaError_t launch_adj(const AdjArgs<T> &a, int N, int v, int C, int grid, int nt, size_t smem, cudaStream_t s) {
  const void *fn = adj_ptr<T>(N, v, C);
  if (!fn) return cudaErrorInvalidValue;
  if (grid <= 0) return cudaSuccess;
  void *args[] = {const_cast<AdjArgs<T> *>(&a)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(nt), args, smem, s);
}

template <typename T>
cudaError_t prepare_adj(int N, int v, int C, size_t smem) {
  const void *fn = adj_ptr<T>(N, v, C);
  if (!fn) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
cudaError_t launch_sqerr(const T *x, const T *xt, long long n, double *part, int blocks, cudaStream_t s) {
  sqerr_kernel<T><<<blocks, 256, 0, s>>>(x, xt, n, part);
  return cudaGetLastError();
}

cudaError_t launch_sum(const double *v, int n, double scale, double *out, cudaStream_t s) {
  sum_kernel<<<1, 256, 0, s>>>(v, n, scale, out);
  return cudaGetLastError();
}

__global__ void add_kernel(double *acc, const double *v) { acc[0] += v[0]; }

cudaError_t launch_add(double *acc, const double *v, cudaStream_t s) {
  add_kernel<<<1, 1, 0, s>>>(acc, v);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_taps(const ImageDesc *desc, int img, int M, int N, int C, int K, const void *G, double *E,
                        void *dh, int accumulate, cudaStream_t s) {
  const int Nh = N / 2 + 1, threads = 32 * (K < 32 ? K : 32);
  taps_stage1_kernel<T><<<Nh, threads, (size_t)M * sizeof(double2), s>>>(
      desc, img, C, K, reinterpret_cast<const cx<T> *>(G), reinterpret_cast<double2 *>(E));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  taps_stage2_kernel<T><<<K, threads, (size_t)N * sizeof(double2), s>>>(
      desc, img, K, reinterpret_cast<const double2 *>(E), reinterpret_cast<T *>(dh), accumulate);
  return cudaGetLastError();
}

#define INST(T)                                                                                                 \
  template cudaError_t launch_adj<T>(const AdjArgs<T> &, int, int, int, int, int, size_t, cudaStream_t);      \
  template cudaError_t prepare_adj<T>(int, int, int, size_t);                                                  \
  template cudaError_t launch_sqerr<T>(const T *, const T *, long long, double *, int, cudaStream_t);          \
  template cudaError_t launch_taps<T>(const ImageDesc *, int, int, int, int, int, const void *, double *, void *, \
                                      int, cudaStream_t);
INST(float)
INST(double)

}  // namespace dcv
