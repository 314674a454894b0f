// Reverse pass (gradient of the unrolled iteration) for the register-FFT
// row lengths L = R V TT (R in {1, 3, 5}).
//
// Reverse of forward step j ((y~_j, v_j, d_j) -> x_{j+1} -> (y~_{j+1},
// v_{j+1}, d_{j+1})), with a = D x_{j+1} + d_j and carried adjoints yb, vb, db:
//   A_j: w = vb - db;  ab = db + J(a) w  (J the Jacobian of vector-soft:
//        (1 - tau/|a|) I + tau a a^T / |a|^3 where |a| > tau, else 0);
//        taub -= a^T w / |a|;  tb = relax M_u yb;  yb' = (M_o - (relax-1) M_u) yb;
//        xb = D^T ab (+ dL/dx at the last step)
//   B_j: bb = (T~^T T~ + mu D^T D)^{-1} (xb + T~^T tb), T~bb   (the forward
//        column pass with the pair (tb, xb) in place of (y~, r))
//   C_j: yb = yb' + T~bb;  vb = mu D bb;  db = ab - mu D bb.
// The kernel below fuses C_{j+1} (it receives bb of step j+1 from the
// column pass and the inverse row DFT) with A_j, and ends with the forward
// row DFT of tb + i xb for B_j.  Per pixel it needs ab of step j at
// (i,p), (i,p-1), (i-1,p) (for D^T), each from bb, x_{j+1} and d_j at three
// points and ab_{j+1} at one, so the CTA stages rows i-1 .. i+1 of bb and
// x_{j+1} and rows i-1 .. i of ab_{j+1} and d_j.
#pragma once

#include "iter_p2.cuh"

namespace dcv {

template <typename T>
__device__ __forceinline__ int find_adj(const ImageDesc *desc, const int *imgs, const int *beg, int n, int wi) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (beg[imgs[mid]] <= wi) lo = mid; else hi = mid - 1;
  }
  return imgs[lo];
}

// V complex values per thread (32: fft_p2, 16: fft_v16); R groups of TT
// threads per (channel, row), each owning L2 = V TT pixels of the row.
template <typename T, int TT, int C, int R, int V>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) row_adj_p2_kernel(AdjArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GS = reg_group_stride<V, TT>(), L2 = V * TT;
  const int wi = blockIdx.x;
  const int img = find_adj<T>(a.desc, a.cls_imgs, a.adj_begin, a.nimg, wi);
  const ImageDesc *Dp = &a.desc[img];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh, Rb = a.rb;
  const int blk = wi - a.adj_begin[img];
  const int r0 = blk * Rb, nr = min(Rb, M - r0);
  const long long P = (long long)M * N, px0 = Dp->px;
  const int g = threadIdx.x / TT, q = threadIdx.x - g * TT;
  const int bar = 1 + g;  // named barrier of a 64-thread group (group_bar)
  const int gr = g % R, row_id = g / R, ch = row_id / Rb, hh = row_id - ch * Rb;
  const bool active = ch < C && hh < nr;
  const int i = r0 + hh;
  const bool start = a.mode == ADJ_START;
  // Staged rows: bb and x (i-1 .. i+1), ab_in and d (i-1 .. i), per channel.
  T *Bs = reinterpret_cast<T *>(smem_raw);                                // [C][Rb+2][N]
  T *Xs = Bs + (size_t)C * (Rb + 2) * N;                                  // [C][Rb+2][N]
  cx<T> *As = reinterpret_cast<cx<T> *>(Xs + (size_t)C * (Rb + 2) * N);   // [C][Rb+1][N]
  cx<T> *Ds = As + (size_t)C * (Rb + 1) * N;                              // [C][Rb+1][N]
  // Per group: tb + i xb, placed beyond both the staged rows and the
  // transpose tiles (the tiles overwrite the staged rows after a barrier).
  const size_t staged = (size_t)C * (2 * (Rb + 2) + 4 * (Rb + 1)) * N * sizeof(T);
  const size_t tiles = (size_t)(blockDim.x / TT) * GS * sizeof(cx<T>);
  cx<T> *Cs = reinterpret_cast<cx<T> *>(smem_raw + (staged > tiles ? staged : tiles)) + (size_t)row_id * N;

  if (!start) {
    for (int c = 0; c < C; ++c) {
      for (int k = 0; k < nr + 2; ++k) {
        const long long ro = px0 + c * P + (long long)wrapi(r0 - 1 + k, M) * N;
        copy_async<T>(Bs + ((size_t)c * (Rb + 2) + k) * N, a.bbuf + ro, N, threadIdx.x, blockDim.x);
        copy_async<T>(Xs + ((size_t)c * (Rb + 2) + k) * N, a.xs + ro, N, threadIdx.x, blockDim.x);
      }
      for (int k = 0; k < nr + 1; ++k) {
        const long long ro = px0 + c * P + (long long)wrapi(r0 - 1 + k, M) * N;
        copy_async<cx<T>>(As + ((size_t)c * (Rb + 1) + k) * N, reinterpret_cast<const cx<T> *>(a.ab_in) + ro, N,
                          threadIdx.x, blockDim.x);
        copy_async<cx<T>>(Ds + ((size_t)c * (Rb + 1) + k) * N, reinterpret_cast<const cx<T> *>(a.ds) + ro, N,
                          threadIdx.x, blockDim.x);
      }
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();

  const T mu = a.mu, tau = a.tau, relax = a.relax;
  T taub = T(0);
  cx<T> *__restrict__ abo = reinterpret_cast<cx<T> *>(a.ab_out);
  if (active) {
    const long long rowp = px0 + ch * P + (long long)i * N;
    const uint32_t *mrow = a.mask + Dp->mask + ch * Dp->mask_plane + (long long)i * (N / 32);
    for (int m = 0; m < V; ++m) {
      const int p = q + TT * m + L2 * gr;
      const int pm = (p == 0) ? N - 1 : p - 1;
      const T yb = start ? T(0) : a.ybar[rowp + p];
      const bool obs = (__ldg(&mrow[p >> 5]) >> (p & 31)) & 1u;
      const T tb = obs ? T(0) : relax * yb;
      a.ybar[rowp + p] = obs ? yb : -(relax - T(1)) * yb;
      T xb;
      if (start) {
        xb = a.xseed ? a.xseed[rowp + p] : a.lscale * (a.xs[rowp + p] - a.xtrue[rowp + p]);
        abo[rowp + p] = mk<T>(T(0), T(0));
      } else {
        // ab_j for channel ch at the points pt = 0: (i, p), 1: (i, p-1), 2: (i-1, p).
        T ab_h0 = T(0), ab_v0 = T(0), ab_h_l = T(0), ab_v_u = T(0);
#pragma unroll
        for (int pt = 0; pt < 3; ++pt) {
          const int rr = (pt == 2) ? hh : hh + 1;      // staged row of the point (hh+1 = row i)
          const int pc = (pt == 1) ? pm : p;
          const int pc1 = (pc + 1 == N) ? 0 : pc + 1;
          T n2 = T(0), aw = T(0), wh_c = T(0), wv_c = T(0), ah_c = T(0), av_c = T(0), dbh_c = T(0), dbv_c = T(0);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const T *br = Bs + ((size_t)c * (Rb + 2) + rr) * N, *xr = Xs + ((size_t)c * (Rb + 2) + rr) * N;
            const cx<T> ain = As[((size_t)c * (Rb + 1) + rr) * N + pc];
            const cx<T> dd = Ds[((size_t)c * (Rb + 1) + rr) * N + pc];
            const T dbh = br[pc1] - br[pc], dbv = br[N + pc] - br[pc];  // D bb
            const T dbar_h = ain.x - mu * dbh, dbar_v = ain.y - mu * dbv;  // db_{j+1}
            const T wh = T(2) * mu * dbh - ain.x, wv = T(2) * mu * dbv - ain.y;  // vb - db
            const T ah = xr[pc1] - xr[pc] + dd.x, av = xr[N + pc] - xr[pc] + dd.y;
            n2 += ah * ah + av * av;
            aw += ah * wh + av * wv;
            if (c == ch) {
              wh_c = wh;
              wv_c = wv;
              ah_c = ah;
              av_c = av;
              dbh_c = dbar_h;
              dbv_c = dbar_v;
            }
          }
          T gh = dbh_c, gv = dbv_c;
          if (n2 > tau * tau) {
            const T rn = rsqrt_t<T>(n2), s1 = T(1) - tau * rn, s2 = tau * aw * rn * rn * rn;
            gh += s1 * wh_c + s2 * ah_c;
            gv += s1 * wv_c + s2 * av_c;
            if (pt == 0 && ch == 0) taub -= aw * rn;
          }
          if (pt == 0) {
            ab_h0 = gh;
            ab_v0 = gv;
          } else if (pt == 1) {
            ab_h_l = gh;
          } else {
            ab_v_u = gv;
          }
        }
        abo[rowp + p] = mk<T>(ab_h0, ab_v0);
        xb = (ab_h_l - ab_h0) + (ab_v_u - ab_v0);
      }
      Cs[p] = mk<T>(tb, xb);
    }
  }
  __syncthreads();  // tiles below reuse the staged rows
  cx<T> v[V];
  if (active) {
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = Cs[R * (q + TT * m) + gr];
  }
  if (R > 1) __syncthreads();  // every group has read its inputs before the combine overwrites Cs
  {
    cx<T> *tile = reinterpret_cast<cx<T> *>(smem_raw) + (size_t)g * GS;
    const unsigned gm = group_mask(TT);
    const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw2);
    fft_reg_smem<T, V, TT, R, -1>(v, active, tile, q, gm, bar, gr, tw + (V == 32 ? Dp->tw2_row : Dp->tw16_row),
                                  tw + Dp->tw3_row, tw + Dp->twab_row, Cs);
    if (R == 1 && active) group_bar<TT>(gm, bar);
  }
  if (active) {
    cpair<T> *dst = a.S_out + Dp->spec + ((long long)ch * M + i) * Nh;
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
  double t = double(taub), z0 = 0.0, z1 = 0.0;
  block_sum3_dyn(t, z0, z1);
  if (threadIdx.x == 0) a.tpart[wi] = t;
}

// Sum over pixels of (x - x_true)^2: per-CTA partial sums (fixed order).
template <typename T>
__global__ void sqerr_kernel(const T *x, const T *xt, long long n, double *part) {
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const T d = x[e] - xt[e];
    s += double(d * d);
  }
  double z0 = 0.0, z1 = 0.0;
  block_sum3_dyn(s, z0, z1);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Fixed-order sum of n doubles into out[0] (one CTA).
static __global__ void sum_kernel(const double *v, int n, double scale, double *out) {
  double s = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) s += v[e];
  double z0 = 0.0, z1 = 0.0;
  block_sum3_dyn(s, z0, z1);
  if (threadIdx.x == 0) out[0] = s * scale;
}

// dL/dh from the accumulated spectrum G (per image and channel, M x (N/2+1)):
// dL/dh[p+b][q+b] = (1/(MN)) sum_k w(k2) Re(G(k) exp(2 pi i (k1 p/M + k2 q/N))),
// w = 1 at k2 = 0 and N/2, 2 elsewhere (G of real correlations is Hermitian).
// Sums in FP64; the roots of unity come from a per-block table built with
// sincospi.  Warp-shuffle reductions, one warp per output.
//
// Stage 1: E(p, k2) = sum_c sum_k1 G_c(k1, k2) exp(2 pi i k1 p / M).  One
// block per k2, warps over p, lanes over k1.
template <typename T>
__global__ void taps_stage1_kernel(const ImageDesc *desc, int img, int C, int K, const cx<T> *G, double2 *E) {
  extern __shared__ double2 rootM[];  // exp(2 pi i j / M), j < M
  const ImageDesc &D = desc[img];
  const int M = D.M, Nh = D.Nh, b = K / 2;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)j / (double)M, &sn, &cs);
    rootM[j] = make_double2(cs, sn);
  }
  __syncthreads();
  const int k2 = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int pi = warp; pi < K; pi += nw) {
    const int p = pi - b, pm = ((p % M) + M) % M;
    double re = 0.0, im = 0.0;
    for (int c = 0; c < C; ++c) {
      const cx<T> *Gc = G + D.spec + (long long)c * M * Nh + k2;
      int ph = (int)(((long long)lane * pm) % M);
      const int step = (int)((32LL * pm) % M);
      for (int k1 = lane; k1 < M; k1 += 32) {
        const cx<T> gv = Gc[(long long)k1 * Nh];
        const double2 w = rootM[ph];
        re += double(gv.x) * w.x - double(gv.y) * w.y;
        im += double(gv.x) * w.y + double(gv.y) * w.x;
        ph += step;
        if (ph >= M) ph -= M;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) E[pi * Nh + k2] = make_double2(re, im);
  }
}

// Stage 2: dh[p][q] (+)= (1/(MN)) sum_k2 w(k2) Re(E(p, k2) exp(2 pi i k2 q / N)).
// One block per p, warps over q, lanes over k2.
template <typename T>
__global__ void taps_stage2_kernel(const ImageDesc *desc, int img, int K, const double2 *E, T *dh, int accumulate) {
  extern __shared__ double2 rootN[];  // exp(2 pi i j / N), j < N
  const ImageDesc &D = desc[img];
  const int N = D.N, Nh = D.Nh, b = K / 2;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)j / (double)N, &sn, &cs);
    rootN[j] = make_double2(cs, sn);
  }
  __syncthreads();
  const int pi = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int qi = warp; qi < K; qi += nw) {
    const int q = qi - b, qm = ((q % N) + N) % N;
    double acc = 0.0;
    int ph = (int)(((long long)lane * qm) % N);
    const int step = (int)((32LL * qm) % N);
    for (int k2 = lane; k2 < Nh; k2 += 32) {
      const double wgt = (k2 == 0 || 2 * k2 == N) ? 1.0 : 2.0;
      const double2 ev = E[pi * Nh + k2], w = rootN[ph];
      acc += wgt * (ev.x * w.x - ev.y * w.y);
      ph += step;
      if (ph >= N) ph -= N;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double sres = acc / ((double)D.M * (double)N);
      const int e = pi * K + qi;
      dh[e] = accumulate ? dh[e] + (T)sres : (T)sres;
    }
  }
}

}  // namespace dcv
