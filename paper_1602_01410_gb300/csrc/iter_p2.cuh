// Row and column passes for the register-transform lengths L = R V TT
// (R in {1, 3, 5}; V = 32 values per thread with fft_p2 / fft_mixed, or
// V = 16 with fft_v16; see fft.cuh).  Same arithmetic as the generic passes
// in iter_kernels.cuh (see the comment there for the iteration), different
// work decomposition:
//
//   row pass:    R groups of TT threads per (channel, row) of the block; each
//                thread owns the pixels q + TT m (+ L/R of its sub-transform)
//                of its row, in registers through the transform.  Inverse
//                half (row_inv_p2_kernel) and forward half (row_fwd_p2_kernel,
//                or its staged variant) are separate kernels, so the forward
//                half's stencil sees the x rows of its neighbours.
//   column pass: R groups per signal (Y or R of one spectral column); the
//                column tile is staged through shared memory with coalesced
//                row loads and stores and transformed in place.
#pragma once

#include "bulk.cuh"
#include "fft.cuh"
#include "internal.h"
#include "iter_kernels.cuh"

namespace dcv {

__device__ __forceinline__ unsigned group_mask(int TT) {
  if (TT >= 32) return 0xffffffffu;
  const int base = (threadIdx.x & 31) / TT * TT;
  return ((1u << TT) - 1u) << base;
}

// Asynchronous global -> shared copies (sm_80+ cp.async), B = 4, 8 or 16 bytes.
template <int B>
__device__ __forceinline__ void cp_async(void *sdst, const void *gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Cooperative asynchronous copy of n elements (4, 8 or 16 bytes each) from
// global to shared memory: 16-byte chunks when both ends are 16-byte aligned.
template <typename E>
__device__ __forceinline__ void copy_async(E *sdst, const E *gsrc, int n, int tid, int nthr) {
  if (sizeof(E) < 16 && (((uintptr_t)gsrc | (uintptr_t)sdst) & 15) == 0 && (n * (int)sizeof(E)) % 16 == 0) {
    const int n16 = n * (int)sizeof(E) / 16;
    for (int k = tid; k < n16; k += nthr)
      cp_async<16>(reinterpret_cast<char *>(sdst) + 16 * k, reinterpret_cast<const char *>(gsrc) + 16 * k);
  } else {
    for (int k = tid; k < n; k += nthr) cp_async<sizeof(E)>(sdst + k, gsrc + k);
  }
}

// Register-transform helpers for V = 32 (fft_p2 / fft_mixed) or V = 16
// (fft_v16, R = 1) values per thread.
template <int V, int TT> __device__ __forceinline__ int reg_pos(int q, int j) {
  if constexpr (V == 32)
    return q + TT * p2_slot<TT>(j);
  else
    return v16_pos<TT>(q, j);
}
template <int V, int TT> __host__ __device__ constexpr int reg_group_stride() {
  return V == 32 ? p2_group_stride<TT>() : v16_group_stride<TT>();
}
// tw2: the [k1][t] table of the sub-length (V = 32) or the [k1][q] table of
// fft_v16 (V = 16); twab: fft_v16's [a][c] table; tw3: the [r][k2] table of
// the radix-R combine (R > 1, both V).
template <typename T, int V, int TT, int R, int SIGN>
__device__ __forceinline__ void fft_reg(cx<T> (&v)[V], bool active, cx<T> *tile, int q, unsigned gm, int bar, int gr,
                                        const cx<T> *__restrict__ tw2, const cx<T> *__restrict__ tw3,
                                        const cx<T> *__restrict__ twab, cx<T> *E) {
  if constexpr (V == 32) {
    fft_mixed<T, TT, R, SIGN>(v, active, tile, q, gm, gr, tw2, tw3, E);
  } else {
    if (active) fft_v16<T, TT, SIGN>(v, tile, q, gm, bar, tw2, twab);
    if constexpr (R > 1) {  // radix-R combine of the R sub-transforms (as in fft_mixed)
      constexpr int L2 = 16 * TT;
      __syncthreads();  // E may overlay the transpose tiles of the other groups
      if (active) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int k2 = v16_pos<TT>(q, j);
          cx<T> w = __ldg(&tw3[gr * L2 + k2]);
          if (SIGN > 0) w.y = -w.y;
          E[gr * L2 + k2] = cmul<T>(v[j], w);
        }
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int k2 = v16_pos<TT>(q, j);
          cx<T> acc = E[k2];
#pragma unroll
          for (int r = 1; r < R; ++r) acc = cadd<T>(acc, cmul<T>(E[r * L2 + k2], root_r<T, R, SIGN>((r * gr) % R)));
          v[j] = acc;
        }
      }
      __syncthreads();
    }
  }
}

// The transform of fft_reg with its result left in shared memory, in
// natural order (E[k] = X[k], k < L), instead of in registers, for passes
// that store the transformed line to shared memory anyway.  For R > 1 the
// radix-R combine runs in place over E: the R TT threads of this transform
// take the L2 positions k2 in turn, read E[r L2 + k2] for every r, apply
// an R-point DFT in registers and write the R outputs back to the same
// places (R reads and R writes per k2, where the register form reads all R
// inputs once per output).  Contains __syncthreads when R > 1 (every thread
// of the CTA calls it); for R = 1 the caller synchronises before reading E.
template <typename T, int V, int TT, int R, int SIGN>
__device__ __forceinline__ void fft_reg_smem(cx<T> (&v)[V], bool active, cx<T> *tile, int q, unsigned gm, int bar,
                                             int gr, const cx<T> *__restrict__ tw2, const cx<T> *__restrict__ tw3,
                                             const cx<T> *__restrict__ twab, cx<T> *E) {
  constexpr int L2 = V * TT;
  if (active) {
    if constexpr (V == 32)
      fft_p2<T, TT, SIGN>(v, tile, q, gm, tw2);
    else
      fft_v16<T, TT, SIGN>(v, tile, q, gm, bar, tw2, twab);
  }
  if constexpr (R == 1) {
    if (active) {
#pragma unroll
      for (int j = 0; j < V; ++j) E[reg_pos<V, TT>(q, j)] = v[j];
    }
  } else {
    __syncthreads();  // E may overlay the transpose tiles of the other groups
    if (active) {
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const int k2 = reg_pos<V, TT>(q, j);
        cx<T> w = __ldg(&tw3[gr * L2 + k2]);
        if (SIGN > 0) w.y = -w.y;
        E[gr * L2 + k2] = cmul<T>(v[j], w);
      }
    }
    __syncthreads();
    if (active) {
      for (int k2 = gr * TT + q; k2 < L2; k2 += R * TT) {
        cx<T> e[R];
#pragma unroll
        for (int r = 0; r < R; ++r) e[r] = E[r * L2 + k2];
        Dft<T, R, SIGN>::run(e);
#pragma unroll
        for (int r = 0; r < R; ++r) E[r * L2 + k2] = e[r];
      }
    }
    __syncthreads();
  }
}

// Register cap of the row kernels: three-channel FP32 rows with 16 values
// per thread (3 R TT threads per pixel row) are held to 72 registers for
// R = 3, 5 (so that three 288-thread CTAs fit one SM's 64 K registers) and
// to 96 for R = 1 (two CTAs of two 1024-point rows; tighter caps spill).
// (The inverse half and the y~ spectrum need fewer: 64 for R = 1.)
template <typename T, int C, int R, int V, bool FWD = true> __host__ __device__ constexpr int row_reg_cap() {
  return (C == 3 && V == 16 && sizeof(T) == 4) ? (R == 1 ? (FWD ? 96 : 64) : 72) : (sizeof(T) == 4 ? 128 : 255);
}

// All three kernels below handle L = R * 32 * TT (R in {1, 3, 5}): a
// transform of length L is done by R groups of TT threads (fft_mixed); with
// R = 1 it is fft_p2 alone.  Work item layout: group g of a CTA serves
// (channel ch, row hh) = (g / R) split as ch = (g / R) / Rb, hh = (g / R) % Rb,
// and sub-transform gr = g % R.

// ----------------------------------------------------------- row (R1) ---
// Inverse half of the row pass: Rb rows per CTA, no halo.  Inverse row DFT
// of X + i HX -> x, T~x; z-update of y~; x to the plan's x buffer (read by
// R2) and optionally to x_out.  The rows' spectra arrive in shared memory
// by bulk copies (one per row, the TMA engine, completed on an mbarrier
// with a bounded wait); the CTA's y~ rows and mask words are staged with
// cp.async while the transforms run.  Statistics:
// ||dz||^2 and the data-fit half of the objective.  ROW_ADJ (reverse pass):
// xbuf <- b, yt <- yt + T~b instead of the z-update.
// Shared memory: [one region of R transpose tiles per (channel, row), which
// the R groups also use as their exchange buffer][y~ C x Rb x N][mask words].
template <typename T, int TT, int C, int R, int V>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) __maxnreg__((row_reg_cap<T, C, R, V, false>())) row_inv_p2_kernel(RowArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GS = reg_group_stride<V, TT>(), L2 = V * TT, RS = R * GS;
  const int wi = blockIdx.x;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, true)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh, Rb = Dp->Rb, wpr = N / 32;
  const int blk = wi - Dp->row_begin;
  const int r0 = blk * Rb, nr = min(Rb, M - r0);
  const long long P = (long long)M * N, px0 = Dp->px;
  const int g = threadIdx.x / TT, q = threadIdx.x - g * TT;
  const int bar = 1 + g;  // named barrier of a 64-thread group (group_bar)
  const int gr = g % R, row_id = g / R, ch = row_id / Rb, hh = row_id - ch * Rb;
  const bool active = ch < C && hh < nr;
  const int i = r0 + hh;
  const bool init = a.mode == ROW_INIT;
  const bool adj = a.mode == ROW_ADJ;      // reverse pass: xbuf <- b, yt <- yt + T~b
  const unsigned gm = group_mask(TT);
  // Distinct buffers (x_out is written only when it is not the x buffer).
  T *__restrict__ yt = a.yt;
  T *__restrict__ xbuf = a.xbuf;
  T *__restrict__ xout = (a.x_out && a.x_out != a.xbuf) ? a.x_out : nullptr;
  cx<T> *Ex = reinterpret_cast<cx<T> *>(smem_raw) + (size_t)row_id * RS;  // this row's region
  cx<T> *tile = Ex + gr * GS;
  T *Ys = reinterpret_cast<T *>(reinterpret_cast<cx<T> *>(smem_raw) + (size_t)C * Rb * RS);  // [C][Rb][N]
  uint32_t *Ms = reinterpret_cast<uint32_t *>(Ys + (size_t)C * Rb * N);              // [C][Rb][N/32]
  const cx<T> *tw2 = reinterpret_cast<const cx<T> *>(a.tw2) + (V == 32 ? Dp->tw2_row : Dp->tw16_row);
  const cx<T> *tw3 = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->tw3_row;
  const cx<T> *twab = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->twab_row;
  // The row spectra (N/2 + 1 pairs, contiguous) arrive in the rows' regions
  // by bulk copies, one per (channel, row); each region holds them (RS >= N
  // + 2 elements) and starts on a 16-byte boundary.
  static_assert(RS >= R * V * TT + 2 && (RS * sizeof(cx<T>)) % 16 == 0, "row region holds the row spectrum");
  __shared__ uint64_t spec_bar;  // completion of the spectra's bulk copies
  const bool spec_in = !init;    // iteration and reverse modes transform the row spectra

  griddep_wait();
  if (spec_in && threadIdx.x == 0) {
    const unsigned row_bytes = (unsigned)(Nh * sizeof(cpair<T>));
    mbar_init(&spec_bar);
    mbar_arrive_expect_tx(&spec_bar, row_bytes * (unsigned)(C * nr));
    for (int c = 0; c < C; ++c)
      for (int h = 0; h < nr; ++h)
        bulk_g2s(reinterpret_cast<cx<T> *>(smem_raw) + (size_t)(c * Rb + h) * RS,
                 a.S_in + Dp->spec + ((long long)c * M + r0 + h) * Nh, row_bytes, &spec_bar);
  }
  if (!init && !adj) {
    for (int c = 0; c < C; ++c) {
      copy_async<T>(Ys + (size_t)c * Rb * N, yt + px0 + c * P + (long long)r0 * N, nr * N, threadIdx.x, blockDim.x);
      copy_async<uint32_t>(Ms + (size_t)c * Rb * wpr, a.mask + Dp->mask + c * Dp->mask_plane + (long long)r0 * wpr,
                           nr * wpr, threadIdx.x, blockDim.x);
    }
  }
  cp_async_commit();
  if (spec_in) {
    __syncthreads();  // the barrier's initialisation is visible to every thread
    const bool ok = mbar_wait(&spec_bar, 0, a.wait_ns);
    if (!__syncthreads_and(ok)) {  // uniform: the whole CTA leaves, its rows untouched
      if (threadIdx.x == 0) {
        atomicOr(a.err, 2);
        (void)mbar_wait(&spec_bar, 0, kDrainNs);  // the copies still in flight land before the block leaves
      }
      cp_async_wait_all();
      return;
    }
  }

  const bool stats = a.partials != nullptr;  // per-thread partials in T, FP64 only for the reduction
  T s_dz = T(0), s_fit = T(0);
  cx<T> v[V];
  const long long rowp = px0 + ch * P + (long long)i * N;
  if (active) {
    if (init) {
#pragma unroll
      for (int j = 0; j < V; ++j) v[j] = mk<T>(yt[rowp + reg_pos<V, TT>(q, j) + L2 * gr], T(0));
    } else {
      const cpair<T> *src = reinterpret_cast<const cpair<T> *>(Ex);
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const int n = R * (q + TT * m) + gr;
        const cpair<T> c = src[2 * n <= N ? n : N - n];
        v[m] = 2 * n <= N ? mk<T>(c.ar - c.bi, c.ai + c.br) : mk<T>(c.ar + c.bi, c.br - c.ai);
      }
    }
  }
  if (!init) {
    // every group of the row has read the spectrum before the tiles overwrite it
    if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
    fft_reg<T, V, TT, R, +1>(v, active, tile, q, gm, bar, gr, tw2, tw3, twab, Ex);
  }
  cp_async_wait_all();
  __syncthreads();
  if (active && adj) {
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int p = reg_pos<V, TT>(q, j) + L2 * gr;
      xbuf[rowp + p] = v[j].x;
      yt[rowp + p] += v[j].y;
    }
  } else if (active) {
    const T relax = a.relax;
    const T *yrow = Ys + ((size_t)ch * Rb + hh) * N;
    const uint32_t *mrow = Ms + ((size_t)ch * Rb + hh) * wpr;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int p = reg_pos<V, TT>(q, j) + L2 * gr;
      xbuf[rowp + p] = v[j].x;
      if (xout) xout[rowp + p] = v[j].x;
      if (!init) {
        const T yo = yrow[p];
        if (!((mrow[p >> 5] >> (p & 31)) & 1u)) {
          const T yn = relax * v[j].y - (relax - T(1)) * yo;
          yt[rowp + p] = yn;
          if (stats) s_dz += (yn - yo) * (yn - yo);
        } else if (stats) {
          s_fit += (yo - v[j].y) * (yo - v[j].y);
        }
      }
    }
  }
  if (stats) {
    double fit = 0.5 * double(s_fit), z = 0.0, dz = double(s_dz);
    block_sum3_dyn(z, dz, fit);
    if (threadIdx.x == 0) {
      double *o = a.partials + 3 * (long long)(Dp->row_pbase + blk);
      o[1] = dz;
      o[2] = fit;
    }
  }
}

// ------------------------------------------------- row, y~ spectrum ---
// Inner block-Gauss-Seidel pass / Tikhonov step, after the inverse half
// updated z: the forward row DFT of y~ alone (real input, so its spectrum is
// Y_row, Hermitian; k <= N/2 is stored into the Y half of S_out, the R half
// is kept).  Same CTA layout as the inverse half; shared memory: one region
// of R transpose tiles per (channel, row).
template <typename T, int TT, int C, int R, int V>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) __maxnreg__((row_reg_cap<T, C, R, V, false>())) row_yspec_p2_kernel(RowArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GS = reg_group_stride<V, TT>(), L2 = V * TT, RS = R * GS;
  const int wi = blockIdx.x;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, true)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh, Rb = Dp->Rb;
  const int blk = wi - Dp->row_begin;
  const int r0 = blk * Rb, nr = min(Rb, M - r0);
  const long long P = (long long)M * N, px0 = Dp->px;
  const int g = threadIdx.x / TT, q = threadIdx.x - g * TT;
  const int bar = 1 + g;  // named barrier of a 64-thread group (group_bar)
  const int gr = g % R, row_id = g / R, ch = row_id / Rb, hh = row_id - ch * Rb;
  const bool active = ch < C && hh < nr;
  const int i = r0 + hh;
  const unsigned gm = group_mask(TT);
  cx<T> *Ex = reinterpret_cast<cx<T> *>(smem_raw) + (size_t)row_id * RS;
  cx<T> *tile = Ex + gr * GS;
  const cx<T> *tw2 = reinterpret_cast<const cx<T> *>(a.tw2) + (V == 32 ? Dp->tw2_row : Dp->tw16_row);
  const cx<T> *tw3 = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->tw3_row;
  const cx<T> *twab = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->twab_row;
  griddep_wait();
  cx<T> v[V];
  if (active) {
    const T *__restrict__ yrow = a.yt + px0 + ch * P + (long long)i * N;
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = mk<T>(yrow[R * (q + TT * m) + gr], T(0));
  }
  fft_reg<T, V, TT, R, -1>(v, active, tile, q, gm, bar, gr, tw2, tw3, twab, Ex);
  if (active) {
    cpair<T> *dst = a.S_out + Dp->spec + ((long long)ch * M + i) * Nh;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int k = reg_pos<V, TT>(q, j) + L2 * gr;
      if (2 * k <= N) *reinterpret_cast<cx<T> *>(&dst[k]) = v[j];
    }
  }
}

// The prox/dual step in explicitly rounded operations: every kernel that
// evaluates it (the row kernels, their staged and fused variants) gets the
// same bits, whatever multiply-adds the compiler would otherwise contract.
template <typename T> struct Rn;
template <> struct Rn<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Rn<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};
// |(a, b)|^2
template <typename T> __device__ __forceinline__ T sq2(T a, T b) { return Rn<T>::fma(a, a, Rn<T>::mul(b, b)); }
// shrinkage factor of the (vectorial) TV prox at squared norm s: max(0, 1 - tau / sqrt(s))
template <typename T> __device__ __forceinline__ T shrink_g(T s, T tau, T tau2) {
  return s > tau2 ? Rn<T>::fma(-tau, rsqrt_t<T>(s), T(1)) : T(0);
}
// one component of d^{k+1} = (1 - g) a
template <typename T> __device__ __forceinline__ T prox_d(T g, T a) { return Rn<T>::mul(Rn<T>::add(T(1), -g), a); }
// r = mu D^T (v - d^{k+1}) at (f,p) from (2g - 1) a at (f,p-1), (f,p), (f-1,p):
// mu ((2 gl - 1) ahl - (2 g0 - 1) ah0 + (2 gu - 1) avu - (2 g0 - 1) av0)
template <typename T> __device__ __forceinline__ T prox_r(T mu, T gl, T ahl, T g0, T ah0, T gu, T avu, T av0) {
  const T w0 = Rn<T>::fma(T(2), g0, T(-1)), wl = Rn<T>::fma(T(2), gl, T(-1)), wu = Rn<T>::fma(T(2), gu, T(-1));
  const T h = Rn<T>::fma(wl, ahl, -Rn<T>::mul(w0, ah0)), v = Rn<T>::fma(wu, avu, -Rn<T>::mul(w0, av0));
  return Rn<T>::mul(mu, Rn<T>::add(h, v));
}

// L2 prefetch of every row the forward half of rows f0 .. f0 + nrows - 1
// reads, every channel: x on rows f0 - 1 .. f0 + nrows (periodic), d on rows
// f0 - 1 .. f0 + nrows - 1 (unless init), y~ on rows f0 .. f0 + nrows - 1.
// Issued by the lanes of warp 0, one bulk prefetch per row, so that the
// loads of the block's later pixels find their rows in L2.  A row need not
// start on a 16-byte boundary (the images before it in the batch can have
// any size); bulk_prefetch_l2 widens each span to whole 16-byte granules,
// which stay inside the plan's 256-byte aligned, padded buffers.
template <typename T, int C, class XRow>
__device__ __forceinline__ void prefetch_fwd_rows(const XRow &xrow, const cx<T> *dg, const T *yg, long long P, int M,
                                                  int N, int f0, int nrows, bool init) {
  if (threadIdx.x >= 32) return;
  const int nx = nrows + 2, nd = init ? 0 : nrows + 1, per = nx + nd + nrows;
  for (int t = threadIdx.x; t < C * per; t += 32) {
    const int c = t / per, r = t - c * per;
    if (r < nx) {
      const int row = (f0 - 1 + r + M) % M;
      bulk_prefetch_l2(xrow(c, row), N * sizeof(T));
    } else if (r < nx + nd) {
      const int row = (f0 - 1 + (r - nx) + M) % M;
      bulk_prefetch_l2(dg + c * P + (long long)row * N, N * sizeof(cx<T>));
    } else {
      bulk_prefetch_l2(yg + c * P + (long long)(f0 + r - nx - nd) * N, N * sizeof(T));
    }
  }
}

// ------------------------------------------- forward half, prox step ---
// Prox/dual step of a plain iteration's forward half (fixed penalty, no
// statistics) for rows f0 .. f0 + nrows - 1 of one image, every channel,
// pixel-major: a full warp takes a run of 32 pixels of one row, each lane
// one pixel and all C channels of it, so the squared norm over channels of
// the vectorial TV prox stays in the thread.  Per channel and pixel:
//   a = D x + d,  g = max(0, 1 - tau / |a|)  (|a| over channels),
//   d^{k+1} = (1 - g) a,  r = mu D^T (v - d^{k+1}) with v - d^{k+1} = (2g - 1) a,
// with D the periodic forward differences (a_h = x(f,p+1) - x(f,p) + d_h,
// a_v = x(f+1,p) - x(f,p) + d_v), so r at (f,p) needs a and g at (f,p),
// (f,p-1) and (f-1,p).  The values at p-1 and p+1 come from the adjacent
// lanes; at the ends of a run, lane c < C reads channel c's pixels just
// outside it and passes them on.  Each input is read once per run: x on
// rows f-1, f, f+1, d on rows f-1 and f, y~ on row f.  Writes d^{k+1} and
// leaves y~ + i r of channel c, row f0 + j at reg0[c cstride + j rstride + p].
// Every lane of a warp runs the same iterations (N is a multiple of 32);
// the threads of a partial last warp take no run.  init: d = 0, g = 1.
// stats: adds ||d^{k+1} - d^k||^2 of its pixels to s_dd and their TV,
// sum_p sqrt(sum_c |D x|^2), to s_tv (per-thread partials).
// Returns false if some r or y~ is not finite.
template <typename T, int C, class XRow>
__device__ __forceinline__ bool prox_rows_pm(const XRow &xrow, const cx<T> *__restrict__ dg,
                                             const T *__restrict__ yg, cx<T> *__restrict__ dout, long long P, int M,
                                             int N, int f0, int nrows, bool init, T tau, T mu, cx<T> *reg0,
                                             size_t cstride, size_t rstride, bool stats, T &s_dd, T &s_tv) {
  static_assert(C >= 1 && C <= 32, "one lane per channel at the ends of a run");
  constexpr unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5, runs = N >> 5;
  const int ce = lane < C ? lane : 0;
  const T tau2 = tau * tau;
  bool finite = true;
  for (int ck = threadIdx.x >> 5; ck < nrows * runs; ck += nw) {
    const int j = ck / runs, base = (ck - j * runs) << 5, p = base + lane;
    const int f = f0 + j, fu = f == 0 ? M - 1 : f - 1, fd = f + 1 == M ? 0 : f + 1;
    const int pl = base == 0 ? N - 1 : base - 1, pe = base + 32 == N ? 0 : base + 32;
    const long long of = (long long)f * N, ofu = (long long)fu * N;
    T x0[C], xd[C], xu[C], yv[C];
    cx<T> d0[C], du[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      x0[c] = xrow(c, f)[p];
      xd[c] = xrow(c, fd)[p];
      xu[c] = xrow(c, fu)[p];
      yv[c] = yg[c * P + of + p];
      d0[c] = init ? mk<T>(T(0), T(0)) : dg[c * P + of + p];
      du[c] = init ? mk<T>(T(0), T(0)) : dg[c * P + ofu + p];
    }
    // channel ce's pixels just outside the run: (f, pl), (f+1, pl), (f, pe), (f-1, pe)
    T lx = T(0), lxd = T(0), rx = T(0), rxu = T(0);
    cx<T> dl = mk<T>(T(0), T(0));
    if (lane < C) {
      lx = xrow(ce, f)[pl];
      lxd = xrow(ce, fd)[pl];
      rx = xrow(ce, f)[pe];
      rxu = xrow(ce, fu)[pe];
      if (!init) dl = dg[ce * P + of + pl];
    }
    T s0 = T(0), su = T(0), tv = T(0), ah0[C], av0[C], avu[C];
    T el_h = T(0), el_n = T(0);  // on lane c: a_h and |a_c|^2 of channel c at (f, pl)
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T xb = __shfl_sync(full, x0[c], 0);  // x(c, f, base)
      T xr1 = __shfl_down_sync(full, x0[c], 1), xu1 = __shfl_down_sync(full, xu[c], 1);
      const T erx = __shfl_sync(full, rx, c), erxu = __shfl_sync(full, rxu, c);
      if (lane == 31) {
        xr1 = erx;
        xu1 = erxu;
      }
      const T gh = xr1 - x0[c], gv = xd[c] - x0[c];
      ah0[c] = gh + d0[c].x;
      av0[c] = gv + d0[c].y;
      if (stats) tv += sq2<T>(gh, gv);
      const T ahu = (xu1 - xu[c]) + du[c].x;
      avu[c] = (x0[c] - xu[c]) + du[c].y;
      s0 += sq2<T>(ah0[c], av0[c]);
      su += sq2<T>(ahu, avu[c]);
      if (lane == c) {
        el_h = (xb - lx) + dl.x;
        el_n = sq2<T>(el_h, (lxd - lx) + dl.y);
      }
    }
    T sl = T(0);  // |a|^2 at (f, pl), summed in channel order (lane 0 uses it)
#pragma unroll
    for (int c = 0; c < C; ++c) sl += __shfl_sync(full, el_n, c);
    const T g0 = init ? T(1) : shrink_g<T>(s0, tau, tau2);
    const T gu = init ? T(1) : shrink_g<T>(su, tau, tau2);
    const T gle = init ? T(1) : shrink_g<T>(sl, tau, tau2);
    T gl = __shfl_up_sync(full, g0, 1);
    if (lane == 0) gl = gle;
    if (stats) s_tv += sqrt(tv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      T ahl = __shfl_up_sync(full, ah0[c], 1);
      const T eh = __shfl_sync(full, el_h, c);
      if (lane == 0) ahl = eh;
      const long long o = c * P + of + p;
      const T dnh = prox_d<T>(g0, ah0[c]), dnv = prox_d<T>(g0, av0[c]);
      dout[o] = mk<T>(dnh, dnv);
      if (stats) s_dd += (dnh - d0[c].x) * (dnh - d0[c].x) + (dnv - d0[c].y) * (dnv - d0[c].y);
      const T r = prox_r<T>(mu, gl, ahl, g0, ah0[c], gu, avu[c], av0[c]);
      finite = finite && isfinite(r) && isfinite(yv[c]);
      reg0[c * cstride + j * rstride + p] = mk<T>(yv[c], r);
    }
  }
  return finite;
}

// ----------------------------------------------------------- row (R2) ---
// Forward half.  When the plan's state exceeds L2, warp 0 first prefetches
// the block's input rows into L2 (prefetch_fwd_rows).  Several channels,
// fixed penalty: the pixel-major prox step (prox_rows_pm).  Otherwise each
// thread reads the x, d and y~ values of its own pixels straight from
// global memory (the neighbours at p-1, p+1 and in rows i-1, i+1 are read
// by adjacent lanes and by the CTAs of adjacent rows, so they come from
// L1/L2).  From them: the prox factor g at (i,p), (i,p-1), (i-1,p)
// (norm over channels), d^{i+1} = (1-g) a, r = mu D^T (v - d^{i+1}) with
// v - d^{i+1} = (2g - 1) a; then the forward row DFT of y~ + i r, split into
// (Y_row, R_row).  Statistics: ||dd||^2 and the TV half of the objective.
// Shared memory: one region of R transpose tiles per (channel, row); it
// holds y~ + i r, then the transpose tiles and the exchange buffer, then the
// transformed row.
template <typename T, int TT, int C, int R, bool ADAPT, int V>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) __maxnreg__((row_reg_cap<T, C, R, V>())) row_fwd_p2_kernel(RowArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GS = reg_group_stride<V, TT>(), L2 = V * TT, RS = R * GS;
  const int wi = blockIdx.x;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, true)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh, Rb = Dp->Rb;
  const int blk = wi - Dp->row_begin;
  const int r0 = blk * Rb, nr = min(Rb, M - r0);
  const long long P = (long long)M * N, px0 = Dp->px;
  const int g = threadIdx.x / TT, q = threadIdx.x - g * TT;
  const int bar = 1 + g;  // named barrier of a 64-thread group (group_bar)
  const int gr = g % R, row_id = g / R, ch = row_id / Rb, hh = row_id - ch * Rb;
  const bool active = ch < C && hh < nr;
  const int i = r0 + hh;
  const int iu = i == 0 ? M - 1 : i - 1, id = i + 1 == M ? 0 : i + 1;
  const bool init = a.mode == ROW_INIT || a.mode == ROW_WARM;  // d = 0, v = D x
  const T *__restrict__ xg = a.xbuf + px0;
  const cx<T> *__restrict__ dg = reinterpret_cast<const cx<T> *>(a.d_in) + px0;
  const T *__restrict__ yg = a.yt + px0;
  cx<T> *__restrict__ dout = reinterpret_cast<cx<T> *>(a.d_out);
  cx<T> *Cs = reinterpret_cast<cx<T> *>(smem_raw) + (size_t)row_id * RS;  // this row's region
  cx<T> *tile = Cs + gr * GS;
  const cx<T> *tw2 = reinterpret_cast<const cx<T> *>(a.tw2) + (V == 32 ? Dp->tw2_row : Dp->tw16_row);
  const cx<T> *tw3 = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->tw3_row;
  const cx<T> *twab = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->twab_row;
  const unsigned gm = group_mask(TT);
  auto xrow = [&](int c, int row) -> const T * { return xg + c * P + (long long)row * N; };

  griddep_wait();
  if (a.prefetch) prefetch_fwd_rows<T, C>(xrow, dg, yg, P, M, N, r0, nr, init);
  // Penalty: fixed, or per image (adaptation): tau = lambda / mu^i, r with
  // mu^{i+1} and d^{i+1} rescaled by s (v - s d^{i+1} = ((1+s) g - s) a).
  const bool norms = ADAPT && a.mode == ROW_NORMS;
  T tau = a.tau, mur = a.mu, sc = T(1);
  if (ADAPT) {
    const int img = (int)(Dp - a.desc);
    tau = T(a.lam64 / (norms ? a.mu_img[img] : a.mu_prev_img[img]));
    mur = T(a.mu_img[img]);
    sc = T(a.dscale_img[img]);
  }
  const T tau2 = tau * tau, sc1 = T(1) + sc;
  cx<T> *__restrict__ vb = reinterpret_cast<cx<T> *>(a.vbuf);
  const bool stats = a.partials != nullptr;  // per-thread partials in T, FP64 only for the reduction
  T s_dd = T(0), s_tv = T(0), s_dv = T(0);
  bool finite = true;
  cx<T> v[V];
  // Several channels, fixed penalty: the pixel-major prox step, each input
  // read once per row and the norm over channels summed in the thread.  One
  // channel, or penalty adaptation: every thread evaluates its own (channel,
  // pixel) with the whole neighbourhood over channels (for one channel the
  // neighbours are the adjacent lanes' pixels, L1 hits, and no CTA-wide
  // barrier is needed before the transform).
  static_assert((R * V * TT) % 32 == 0, "the pixel-major step takes whole 32-pixel runs of a row");
  bool pixel_major = false;
  if constexpr (C > 1 && !ADAPT) pixel_major = true;
  if (pixel_major) {
    finite = prox_rows_pm<T, C>(xrow, dg, yg, dout + px0, P, M, N, r0, nr, init, tau, a.mu,
                                reinterpret_cast<cx<T> *>(smem_raw), (size_t)Rb * RS, (size_t)RS, stats, s_dd,
                                s_tv);
  } else if (active) {
#pragma unroll 4
    for (int m = 0; m < V; ++m) {
      const int p = q + TT * m + L2 * gr;
      const int pm = (p == 0) ? N - 1 : p - 1, p1 = (p + 1 == N) ? 0 : p + 1;
      T s0 = T(0), sl = T(0), su = T(0), tv = T(0);
      T ah0 = T(0), av0 = T(0), ahl = T(0), avu = T(0), dh0 = T(0), dv0 = T(0);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T *xr = xg + c * P + (long long)i * N, *xu = xg + c * P + (long long)iu * N,
                *xd = xg + c * P + (long long)id * N;
        const T x0 = xr[p], xl = xr[pm], xrr = xr[p1], xdn = xd[p], xdl = xd[pm], xup = xu[p], xul = xu[p1];
        cx<T> d0 = mk<T>(T(0), T(0)), dl = d0, du = d0;
        if (!init) {
          const cx<T> *dr = dg + c * P + (long long)i * N, *dru = dg + c * P + (long long)iu * N;
          d0 = dr[p];
          dl = dr[pm];
          du = dru[p];
        }
        const T gh = xrr - x0, gv = xdn - x0;
        const T a_h = gh + d0.x, a_v = gv + d0.y;
        s0 += sq2<T>(a_h, a_v);
        tv += sq2<T>(gh, gv);
        const T a_hl = (x0 - xl) + dl.x, a_vl = (xdl - xl) + dl.y;
        sl += sq2<T>(a_hl, a_vl);
        const T a_hu = (xul - xup) + du.x, a_vu = (x0 - xup) + du.y;
        su += sq2<T>(a_hu, a_vu);
        if (c == ch) {
          ah0 = a_h;
          av0 = a_v;
          ahl = a_hl;
          avu = a_vu;
          dh0 = d0.x;
          dv0 = d0.y;
        }
      }
      const T g0 = init ? T(1) : shrink_g<T>(s0, tau, tau2);
      const T gl = init ? T(1) : shrink_g<T>(sl, tau, tau2);
      const T gu = init ? T(1) : shrink_g<T>(su, tau, tau2);
      const T dnh = prox_d<T>(g0, ah0), dnv = prox_d<T>(g0, av0);
      const long long o = px0 + ch * P + (long long)i * N + p;
      if (ADAPT && norms) {
        // residuals of Eq. (varying_penalty): d^{i+1} - d^i and v^{i+1} - v^i
        const cx<T> vo = vb[o], vn = mk<T>(g0 * ah0, g0 * av0);
        s_dd += (dnh - dh0) * (dnh - dh0) + (dnv - dv0) * (dnv - dv0);
        s_dv += (vn.x - vo.x) * (vn.x - vo.x) + (vn.y - vo.y) * (vn.y - vo.y);
        vb[o] = vn;
        continue;
      }
      if (ADAPT) {
        dout[o] = mk<T>(sc * dnh, sc * dnv);
        if (init) vb[o] = mk<T>(g0 * ah0, g0 * av0);  // v^0 = D x^0
      } else {
        dout[o] = mk<T>(dnh, dnv);
      }
      if (stats) {
        s_dd += (dnh - dh0) * (dnh - dh0) + (dnv - dv0) * (dnv - dv0);
        if (ch == 0) s_tv += sqrt(tv);
      }
      const T r = ADAPT ? mur * (((sc1 * gl - sc) * ahl - (sc1 * g0 - sc) * ah0) +
                                 ((sc1 * gu - sc) * avu - (sc1 * g0 - sc) * av0))
                        : prox_r<T>(a.mu, gl, ahl, g0, ah0, gu, avu, av0);
      const T yv = yg[ch * P + (long long)i * N + p];
      finite = finite && isfinite(r) && isfinite(yv);
      Cs[p] = mk<T>(yv, r);
    }
  }
  if (ADAPT && norms) {  // uniform: the whole CTA leaves here
    double dd = double(s_dd), dv = double(s_dv), z = 0.0;
    block_sum3_dyn(dd, dv, z);
    if (threadIdx.x == 0) {
      a.apart[2 * (long long)(Dp->row_pbase + blk)] = dd;
      a.apart[2 * (long long)(Dp->row_pbase + blk) + 1] = dv;
    }
    return;
  }
  if (!finite) atomicOr(a.err, 1);
  // the rows' y~ + i r are in the regions (written by any warp on the plain path)
  if (R > 1 || pixel_major) __syncthreads(); else group_bar<TT>(gm, bar);
  if (active) {
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = Cs[R * (q + TT * m) + gr];
  }
  // every group of the row has read its inputs before the tiles overwrite them
  if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
  fft_reg_smem<T, V, TT, R, -1>(v, active, tile, q, gm, bar, gr, tw2, tw3, twab, Cs);
  if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
  if (active) {
    cpair<T> *__restrict__ dst = a.S_out + Dp->spec + ((long long)ch * M + i) * Nh;
    for (int k = q + TT * gr; k < Nh; k += TT * R) {
      const cx<T> c1 = Cs[k], c2 = Cs[k == 0 ? 0 : N - k];
      cpair<T> o;
      o.ar = T(0.5) * (c1.x + c2.x);
      o.ai = T(0.5) * (c1.y - c2.y);
      o.br = T(0.5) * (c1.y + c2.y);
      o.bi = T(0.5) * (c2.x - c1.x);
      dst[k] = o;
    }
  }
  if (stats) {
    double tvl = double(a.lambda) * double(s_tv), z = 0.0, dd = double(s_dd);
    block_sum3_dyn(dd, z, tvl);
    if (threadIdx.x == 0) {
      double *o = a.partials + 3 * (long long)(Dp->row_pbase + blk);
      o[0] = dd;
      o[2] += tvl;
    }
  }
}

// ------------------------------------------------- row (R2), staged ---
// Forward half, staged variant (used where the staged rows fit: one
// channel).  The CTA stages x (rows r0-1 .. r1), d (rows r0-1 .. r1-1)
// and y~ (rows r0 .. r1-1) of every channel into shared memory with one
// batch of asynchronous copies.  From them: the prox factor g at (i,p),
// (i,p-1), (i-1,p) (norm over channels), d^{i+1} = (1-g) a,
// r = mu D^T (v - d^{i+1}) with v - d^{i+1} = (2g - 1) a; then the forward
// row DFT of y~ + i r, split into (Y_row, R_row).  Statistics: ||dd||^2 and
// the TV half of the objective.
// Shared memory: [x C x (Rb+2) rows][d C x (Rb+1) rows][y~ C x Rb rows] (the
// transpose tiles reuse it after a barrier), then per row y~ + i r and the
// exchange buffer.
template <typename T, int TT, int C, int R, int V>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) row_fwd_p2_staged_kernel(RowArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GS = reg_group_stride<V, TT>(), L2 = V * TT;
  const int wi = blockIdx.x;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, true)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh, Rb = Dp->Rb;
  const int blk = wi - Dp->row_begin;
  const int r0 = blk * Rb, nr = min(Rb, M - r0);
  const long long P = (long long)M * N, px0 = Dp->px;
  const int g = threadIdx.x / TT, q = threadIdx.x - g * TT;
  const int bar = 1 + g;  // named barrier of a 64-thread group (group_bar)
  const int gr = g % R, row_id = g / R, ch = row_id / Rb, hh = row_id - ch * Rb;
  const bool active = ch < C && hh < nr;
  const int i = r0 + hh;
  const bool init = a.mode == ROW_INIT || a.mode == ROW_WARM;  // d = 0, v = D x
  cx<T> *__restrict__ dout = reinterpret_cast<cx<T> *>(a.d_out);
  T *Xs = reinterpret_cast<T *>(smem_raw);                               // [C][Rb+2][N]
  cx<T> *Ds = reinterpret_cast<cx<T> *>(Xs + (size_t)C * (Rb + 2) * N);  // [C][Rb+1][N]
  T *Ys = reinterpret_cast<T *>(Ds + (size_t)C * (Rb + 1) * N);           // [C][Rb][N]
  const size_t staged = (size_t)C * ((Rb + 2) + 2 * (Rb + 1) + Rb) * N * sizeof(T);
  const size_t tiles = (size_t)(blockDim.x / TT) * GS * sizeof(cx<T>);
  cx<T> *Cs = reinterpret_cast<cx<T> *>(smem_raw + (staged > tiles ? staged : tiles)) + (size_t)row_id * N;
  cx<T> *Ex = reinterpret_cast<cx<T> *>(smem_raw + (staged > tiles ? staged : tiles)) + (size_t)C * Rb * N +
              (size_t)row_id * N;
  const cx<T> *tw2 = reinterpret_cast<const cx<T> *>(a.tw2) + (V == 32 ? Dp->tw2_row : Dp->tw16_row);
  const cx<T> *tw3 = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->tw3_row;
  const cx<T> *twab = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->twab_row;

  griddep_wait();
  for (int c = 0; c < C; ++c) {
    for (int k = 0; k < nr + 2; ++k)
      copy_async<T>(Xs + ((size_t)c * (Rb + 2) + k) * N, a.xbuf + px0 + c * P + (long long)wrapi(r0 - 1 + k, M) * N,
                    N, threadIdx.x, blockDim.x);
    if (!init)
      for (int k = 0; k < nr + 1; ++k)
        copy_async<cx<T>>(Ds + ((size_t)c * (Rb + 1) + k) * N,
                          reinterpret_cast<const cx<T> *>(a.d_in) + px0 + c * P + (long long)wrapi(r0 - 1 + k, M) * N,
                          N, threadIdx.x, blockDim.x);
    copy_async<T>(Ys + (size_t)c * Rb * N, a.yt + px0 + c * P + (long long)r0 * N, nr * N, threadIdx.x, blockDim.x);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();

  const T tau = a.tau, tau2 = a.tau * a.tau;
  const bool stats = a.partials != nullptr;  // per-thread partials in T, FP64 only for the reduction
  T s_dd = T(0), s_tv = T(0);
  bool finite = true;
  if (active) {
#pragma unroll 4
    for (int m = 0; m < V; ++m) {
      const int p = q + TT * m + L2 * gr;
      const int pm = (p == 0) ? N - 1 : p - 1, p1 = (p + 1 == N) ? 0 : p + 1;
      T s0 = T(0), sl = T(0), su = T(0), tv = T(0);
      T ah0 = T(0), av0 = T(0), ahl = T(0), avu = T(0), dh0 = T(0), dv0 = T(0);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T *xr = Xs + ((size_t)c * (Rb + 2) + hh + 1) * N;  // row i; xr - N: i-1, xr + N: i+1
        const T x0 = xr[p], xl = xr[pm], xrr = xr[p1], xdn = xr[N + p], xdl = xr[N + pm], xup = xr[p - N],
                xul = xr[p1 - N];
        const cx<T> *dr = Ds + ((size_t)c * (Rb + 1) + hh + 1) * N;  // row i; dr - N: i-1
        const cx<T> d0 = init ? mk<T>(T(0), T(0)) : dr[p];
        const cx<T> dl = init ? mk<T>(T(0), T(0)) : dr[pm];
        const cx<T> du = init ? mk<T>(T(0), T(0)) : dr[p - N];
        const T gh = xrr - x0, gv = xdn - x0;
        const T a_h = gh + d0.x, a_v = gv + d0.y;
        s0 += sq2<T>(a_h, a_v);
        tv += sq2<T>(gh, gv);
        const T a_hl = (x0 - xl) + dl.x, a_vl = (xdl - xl) + dl.y;
        sl += sq2<T>(a_hl, a_vl);
        const T a_hu = (xul - xup) + du.x, a_vu = (x0 - xup) + du.y;
        su += sq2<T>(a_hu, a_vu);
        if (c == ch) {
          ah0 = a_h;
          av0 = a_v;
          ahl = a_hl;
          avu = a_vu;
          dh0 = d0.x;
          dv0 = d0.y;
        }
      }
      const T g0 = init ? T(1) : shrink_g<T>(s0, tau, tau2);
      const T gl = init ? T(1) : shrink_g<T>(sl, tau, tau2);
      const T gu = init ? T(1) : shrink_g<T>(su, tau, tau2);
      const T dnh = prox_d<T>(g0, ah0), dnv = prox_d<T>(g0, av0);
      dout[px0 + ch * P + (long long)i * N + p] = mk<T>(dnh, dnv);
      if (stats) {
        s_dd += (dnh - dh0) * (dnh - dh0) + (dnv - dv0) * (dnv - dv0);
        if (ch == 0) s_tv += sqrt(tv);
      }
      const T r = prox_r<T>(a.mu, gl, ahl, g0, ah0, gu, avu, av0);
      const T yv = Ys[((size_t)ch * Rb + hh) * N + p];
      finite = finite && isfinite(r) && isfinite(yv);
      Cs[p] = mk<T>(yv, r);
    }
  }
  if (!finite) atomicOr(a.err, 1);
  __syncthreads();  // the transpose tiles below reuse the staged rows
  cx<T> v[V];
  if (active) {
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = Cs[R * (q + TT * m) + gr];
  }
  if (R > 1) __syncthreads();  // every group has read its inputs before outputs overwrite Cs
  cx<T> *tile = reinterpret_cast<cx<T> *>(smem_raw) + (size_t)g * GS;
  const unsigned gm = group_mask(TT);
  fft_reg_smem<T, V, TT, R, -1>(v, active, tile, q, gm, bar, gr, tw2, tw3, twab, Cs);
  if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
  if (active) {
    cpair<T> *__restrict__ dst = a.S_out + Dp->spec + ((long long)ch * M + i) * Nh;
    for (int k = q + TT * gr; k < Nh; k += TT * R) {
      const cx<T> c1 = Cs[k], c2 = Cs[k == 0 ? 0 : N - k];
      cpair<T> o;
      o.ar = T(0.5) * (c1.x + c2.x);
      o.ai = T(0.5) * (c1.y - c2.y);
      o.br = T(0.5) * (c1.y + c2.y);
      o.bi = T(0.5) * (c2.x - c1.x);
      dst[k] = o;
    }
  }
  if (stats) {
    double tvl = double(a.lambda) * double(s_tv), z = 0.0, dd = double(s_dd);
    block_sum3_dyn(dd, z, tvl);
    if (threadIdx.x == 0) {
      double *o = a.partials + 3 * (long long)(Dp->row_pbase + blk);
      o[0] = dd;
      o[2] += tvl;
    }
  }
}

// --------------------------------------------------------------- column ---
// One set of R groups per signal (Y or R of one spectral column) of a tile of
// W columns.  The tile is staged with cp.async (coalesced row segments) into
// one shared-memory column per signal; the signal's R groups transform it in
// place (their transpose tiles and exchange buffer are that column's
// storage).  Shared memory: [2W columns of R tiles (+4 elements of padding,
// which spreads the staging stores over the banks)][H^ tile M x w][sin^2 tables].
// FP32 with 16 values per thread: at most 80 registers, so two CTAs of up to
// 384 threads fit one SM (at 86-94 registers the wide column tiles ran one).
template <typename T, int TT, int R, bool EXT, int V>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) __maxnreg__((V == 16 && sizeof(T) == 4) ? 80 : 128)
    col_pass_p2_kernel(ColArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GS = reg_group_stride<V, TT>(), SR = R * GS + 4;
  const int wi = blockIdx.x;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, false)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh;
  const int local = wi - Dp->col_begin;
  const int ch = local / Dp->col_tiles, t = local - ch * Dp->col_tiles;
  const int k20 = t * Dp->W, w = min(Dp->W, Nh - k20);
  const cx<T> *tw2 = reinterpret_cast<const cx<T> *>(a.tw2) + (V == 32 ? Dp->tw2_col : Dp->tw16_col);
  const cx<T> *tw3 = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->tw3_col;
  const cx<T> *twab = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->twab_col;
  const cx<T> *__restrict__ H = reinterpret_cast<const cx<T> *>(a.hhat) + Dp->hhat;
  const T *s2c = a.s2 + Dp->s2_col, *s2r = a.s2 + Dp->s2_row;
  cx<T> *St = reinterpret_cast<cx<T> *>(smem_raw);                  // [2W][SR]
  cx<T> *Hs = St + (size_t)2 * Dp->W * SR;                           // [M][w] H^ tile
  T *S2s = reinterpret_cast<T *>(Hs + (size_t)M * Dp->W);            // [M] column sin^2, then [W] row sin^2
  const int g = threadIdx.x / TT, q = threadIdx.x - g * TT;
  const int bar = 1 + g;  // named barrier of a 64-thread group (group_bar)
  const unsigned gm = group_mask(TT);
  const int gr = g % R, sig = g / R;
  cx<T> *col = St + (size_t)sig * SR;  // this signal's column
  cx<T> *tile = col + gr * GS;
  const long long base = Dp->spec + (long long)ch * M * Nh + k20;
  const int nthr = blockDim.x;

  // Loops below give each thread one signal column s of the tile (s < 2W) and
  // rows r0t, r0t + rstep, ... (nthr is a multiple of 2W), avoiding division.
  const int S2 = 2 * Dp->W, scol = threadIdx.x % S2, r0t = threadIdx.x / S2, rstep = nthr / S2;
  const bool lane_ok = threadIdx.x < rstep * S2;  // threads beyond whole column sets stay idle here
  const bool scol_on = lane_ok && scol < 2 * w;
  griddep_wait();
  if (scol_on)
    for (int ii = r0t; ii < M; ii += rstep)
      cp_async<sizeof(cx<T>)>(&St[scol * SR + ii],
                              reinterpret_cast<const cx<T> *>(&a.S_in[base + (long long)ii * Nh]) + scol);
  if (lane_ok && scol < w)
    for (int k1 = r0t; k1 < M; k1 += rstep) cp_async<sizeof(cx<T>)>(&Hs[k1 * w + scol], &H[(long long)k1 * Nh + k20 + scol]);
  for (int e = threadIdx.x; e < M + w; e += nthr)
    cp_async<sizeof(T)>(&S2s[e], e < M ? &s2c[e] : &s2r[k20 + e - M]);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  cx<T> v[V];
  const bool active = sig < 2 * w;
  if (active) {
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = col[R * (q + TT * m) + gr];
  }
  if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
  fft_reg_smem<T, V, TT, R, -1>(v, active, tile, q, gm, bar, gr, tw2, tw3, twab, col);
  __syncthreads();
  // EXT: a Tikhonov warm-start step (tikh > 0) or a per-image penalty.
  const T mu = (EXT && a.mu_img) ? T(a.mu_img[Dp - a.desc]) : a.mu, tikh = EXT ? a.tikh : T(0);
  const T scale = T(1) / (T(M) * T(N));
  // Solve and store: a full tile (w = W) gives the first (nthr / w) w
  // threads of the CTA a column ww and rows in turn, k1 fastest in the
  // solve (conflict-free column accesses) and ww fastest in the store
  // (whole 32-byte row segments); a ragged tile keeps the staging layout.
  const bool full = w == Dp->W;
  const int kstep = full ? nthr / w : rstep;
  const bool full_on = full && (int)threadIdx.x < kstep * w;
  const int sv_ww = full ? threadIdx.x / kstep : scol, sv_k0 = full ? threadIdx.x % kstep : r0t;
  if (full_on || (!full && lane_ok && scol < w)) {
    const int ww = sv_ww;
    const T s2w = S2s[M + ww];
    cx<T> *gacc = a.gacc ? reinterpret_cast<cx<T> *>(a.gacc) + base : nullptr;
    cx<T> *cy = St + (size_t)(2 * ww) * SR, *cr = cy + SR;
    for (int k1 = sv_k0; k1 < M; k1 += kstep) {
      const cx<T> hv = Hs[k1 * w + ww];
      const T den = hv.x * hv.x + hv.y * hv.y + ((EXT && tikh > T(0)) ? tikh : mu * (S2s[k1] + s2w));
      const T inv = scale / den;
      const cx<T> Y = cy[k1], Rv = (EXT && tikh > T(0)) ? mk<T>(T(0), T(0)) : cr[k1];
      const cx<T> B = cadd<T>(cmulc<T>(hv, Y), Rv);  // den * (solution spectrum)
      if (a.spec_store) {
        cpair<T> o;
        o.ar = Y.x;
        o.ai = Y.y;
        o.br = Rv.x;
        o.bi = Rv.y;
        a.spec_store[base + (long long)k1 * Nh + ww] = o;
      }
      if (gacc) {
        // Reverse pass of the x-step and of T~x (gradient w.r.t. h): with the
        // forward spectra Yf, Rf of this step, Xf = (conj(H) Yf + Rf)/den and
        // the adjoint spectra Tb = Y, Bb = B/den,
        //   G += conj(Bb) (Yf - H Xf) + conj(Xf) (Tb - H Bb).
        const cpair<T> f = a.spec_fwd[base + (long long)k1 * Nh + ww];
        const cx<T> Yf = mk<T>(f.ar, f.ai), Rf = mk<T>(f.br, f.bi);
        const T rden = T(1) / den;
        const cx<T> Xf = cscale<T>(cadd<T>(cmulc<T>(hv, Yf), Rf), rden);
        const cx<T> Bb = cscale<T>(B, rden);
        const cx<T> e1 = csub<T>(Yf, cmul<T>(hv, Xf)), e2 = csub<T>(Y, cmul<T>(hv, Bb));
        cx<T> gv = gacc[(long long)k1 * Nh + ww];
        gv = cadd<T>(gv, cadd<T>(cmulc<T>(Bb, e1), cmulc<T>(Xf, e2)));
        gacc[(long long)k1 * Nh + ww] = gv;
      }
      const cx<T> Xv = cscale<T>(B, inv);
      cy[k1] = Xv;
      cr[k1] = cmul<T>(hv, Xv);
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = col[R * (q + TT * m) + gr];
  }
  if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
  fft_reg_smem<T, V, TT, R, +1>(v, active, tile, q, gm, bar, gr, tw2, tw3, twab, col);
  __syncthreads();
  if (full_on || (!full && lane_ok && scol < w)) {
    const int ww = full ? threadIdx.x % w : scol;
    const cx<T> *cx_ = St + (size_t)(2 * ww) * SR, *ch_ = cx_ + SR;
    for (int ii = full ? threadIdx.x / w : r0t; ii < M; ii += full ? nthr / w : rstep) {
      const cx<T> Xv = cx_[ii], HX = ch_[ii];
      cpair<T> c;
      c.ar = Xv.x;
      c.ai = Xv.y;
      c.br = HX.x;
      c.bi = HX.y;
      a.S_out[base + (long long)ii * Nh + ww] = c;
    }
  }
}

}  // namespace dcv
