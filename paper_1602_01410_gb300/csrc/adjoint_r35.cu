// Reverse-pass row kernels of the lengths 3 * 2^k and 5 * 2^k (16 values per
// thread: L = R * 16 * TT with TT in {8, 16, 32}), in a translation unit of
// their own so that the build compiles them in parallel.
#include "adjoint.cuh"

namespace dcv {

template <typename T, int C, int R>
static const void *adj_r_tt(int tt) {
  switch (tt) {
    case 8: return (const void *)row_adj_p2_kernel<T, 8, C, R, 16>;
    case 16: return (const void *)row_adj_p2_kernel<T, 16, C, R, 16>;
    case 32: return (const void *)row_adj_p2_kernel<T, 32, C, R, 16>;
  }
  return nullptr;
}

template <typename T>
const void *adj_ptr_r35(int N, int v, int C) {
  if (v != 16) return nullptr;
  const int r = N % 3 == 0 ? 3 : (N % 5 == 0 ? 5 : 0);
  if (!r || N % (16 * r) != 0) return nullptr;
  const int tt = N / (16 * r);
  if (r == 3) return C == 3 ? adj_r_tt<T, 3, 3>(tt) : adj_r_tt<T, 1, 3>(tt);
  return C == 3 ? adj_r_tt<T, 3, 5>(tt) : adj_r_tt<T, 1, 5>(tt);
}

template const void *adj_ptr_r35<float>(int, int, int);
template const void *adj_ptr_r35<double>(int, int, int);

}  // namespace dcv
