// The two fused passes of one partial-ADMM iteration.
//
// State per image (Sec. II-B): y~ (observed pixels hold y, unobserved hold
// z), the scaled dual d_x = (d_h, d_v) per pixel, and the row spectra of the
// next x-step's right-hand side.  One iteration i -> i+1 is
//
//   column pass:  forward column DFTs of (Y_row, R_row) -> Y^, R^;
//                 X = (conj(H^) Y^ + R^) / (|H^|^2 + mu (|D^_h|^2 + |D^_v|^2))
//                 (Eq. (dual_x_iter_resolved_boundaries) in the DFT basis),
//                 HX = H^ X;  inverse column DFTs.
//   row pass:     inverse row DFT of X + i HX  ->  x^{i+1} (real part) and
//                 T~ x^{i+1} (imaginary part);
//                 z^{i+1} = relax T~x - (relax - 1) z^i on unobserved pixels
//                 (the over-relaxed Eq. (dual_z_iter_resolved_boundaries));
//                 a = D x + d;  v = vector-soft(a, lambda/mu)   (Eq. (admm_aprox_3), Sec. III-B)
//                 d^{i+1} = a - v                                (Eq. (admm_aprox_4))
//                 r = mu D^T (v - d^{i+1})   (right-hand side of the next x-step)
//                 forward row DFT of y~ + i r, split into (Y_row, R_row).
//
// With g = max(1 - tau/||a||, 0) the prox output is v = g a, so
// d^{i+1} = (1 - g) a and v - d^{i+1} = (2 g - 1) a: only g per pixel must be
// shared between neighbouring pixels (and, for the vectorial TV of
// Sec. III-C, between channels), and a is recomputed from x and d where
// needed.  D uses periodic forward differences and D^T its transpose, so the
// row pass of rows [r0, r1) needs x on rows r0-1 .. r1 (one halo row on each
// side, recomputed by the CTA) and d on rows r0-1 .. r1-1.
#pragma once

#include "fft.cuh"
#include "internal.h"

namespace dcv {

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T> __device__ __forceinline__ T rsqrt_t(T s);
template <> __device__ __forceinline__ float rsqrt_t<float>(float s) { return rsqrtf(s); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double s) { return 1.0 / sqrt(s); }

template <typename T> __device__ __forceinline__ cpair<T> ld_pair(const cpair<T> *p) { return *p; }
template <typename T> __device__ __forceinline__ void st_pair(cpair<T> *p, cpair<T> v) { *p = v; }

__device__ __forceinline__ bool mask_bit(const uint32_t *bits, long long word0, long long idx) {
  return (__ldg(&bits[word0 + (idx >> 5)]) >> (idx & 31)) & 1u;
}

// Image of work item wi within a kernel class (its images in order of
// increasing first work item).
// Programmatic dependent launch: the iteration kernels may be launched while
// their predecessor in the stream is still running (plan option); everything
// before this wait reads only the plan's immutable tables (image
// descriptors, class lists), everything after it may read and write the
// state.  Without the launch attribute it returns at once.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

__device__ __forceinline__ int find_item(const ImageDesc *desc, const int *imgs, int n, int wi, bool row) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    const ImageDesc &D = desc[imgs[mid]];
    if ((row ? D.row_begin : D.col_begin) <= wi) lo = mid; else hi = mid - 1;
  }
  return imgs[lo];
}

// Deterministic CTA reduction of three doubles for any block size that is a
// multiple of 32 (at most 1024); result valid in thread 0.
__device__ __forceinline__ void block_sum3_dyn(double &a, double &b, double &c) {
  __shared__ double red[3][32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = a;
    red[1][w] = b;
    red[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = c = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += red[0][i];
      b += red[1][i];
      c += red[2][i];
    }
  }
}

// Deterministic CTA reduction of three doubles; result valid in thread 0.
template <int NT>
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c) {
  __shared__ double red[3][NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = a;
    red[1][w] = b;
    red[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = c = 0.0;
    for (int i = 0; i < NT / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
      c += red[2][i];
    }
  }
}

// ------------------------------------------------------------------ row ---
// Grid: one CTA per (image, block of Rb rows).  Shared memory: the complex
// row buffer N x ld (ld = (C (Rb+2)) | 1) followed by g for rows r0-1..r1-1.
template <typename T, int NT, int C>
__global__ void __launch_bounds__(NT) row_pass_kernel(RowArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int KMAX = 16 / C;  // owned pixels per thread (host guarantees C*Rb*N <= 16 NT)

  const int wi = blockIdx.x;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, true)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh;
  const int r0 = (wi - Dp->row_begin) * Dp->Rb;
  const int nr = min(Dp->Rb, M - r0);
  const int nh = nr + 2;
  const int S = C * nh, ld = S | 1;
  const long long P = (long long)M * N, px0 = Dp->px, spec0 = Dp->spec;
  const long long mword = Dp->mask, mplane = Dp->mask_plane;
  const FftSched sc = Dp->sched_row;
  const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw) + Dp->tw_row;

  cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
  T *bufr = reinterpret_cast<T *>(smem_raw);  // scalar view: x at 2k, second slot at 2k+1
  T *G = reinterpret_cast<T *>(buf + (size_t)N * ld);
  const bool init = a.mode == ROW_INIT;                            // x = y~0, no z-update
  const bool g_one = init || a.mode == ROW_WARM;                   // initial state: d = 0, v = D x
  const bool inner = a.mode == ROW_INNER;                          // z-update and Y spectrum only
  const cx<T> *din = reinterpret_cast<const cx<T> *>(a.d_in);
  cx<T> *dout = reinterpret_cast<cx<T> *>(a.d_out);

  griddep_wait();
  // 1. rows r0-1 .. r1 of x + i T~x (ROW_ITER: Hermitian-extended inverse
  //    input; ROW_INIT: x^0 = y~0, imaginary part unused).
  if (init) {
    for (int e = threadIdx.x; e < nh * N; e += NT) {
      const int h = e / N, n = e - h * N, i = wrapi(r0 - 1 + h, M);
#pragma unroll
      for (int ch = 0; ch < C; ++ch)
        buf[n * ld + ch * nh + h] = mk<T>(a.yt[px0 + ch * P + (long long)i * N + n], T(0));
    }
  } else {
    for (int e = threadIdx.x; e < nh * Nh; e += NT) {
      const int h = e / Nh, k = e - h * Nh, i = wrapi(r0 - 1 + h, M);
#pragma unroll
      for (int ch = 0; ch < C; ++ch) {
        const cpair<T> q = ld_pair(&a.S_in[spec0 + ((long long)ch * M + i) * Nh + k]);
        const int sg = ch * nh + h;
        buf[k * ld + sg] = mk<T>(q.ar - q.bi, q.ai + q.br);                      // X + i HX
        if (k > 0 && 2 * k != N) buf[(N - k) * ld + sg] = mk<T>(q.ar + q.bi, q.br - q.ai);  // conj(X) + i conj(HX)
      }
    }
  }
  __syncthreads();
  if (!init) fft_smem<T, NT, +1>(buf, N, S, ld, sc, tw);

  // 2. z-update, a = D x + d, g, d^{i+1} (rows r0-1 .. r1-1; updates only on owned rows).
  // Penalty: fixed, or per image (adaptation): tau = lambda / mu^i, r with
  // mu^{i+1} and d^{i+1} rescaled by s (v - s d^{i+1} = ((1+s) g - s) a).
  const bool norms = a.mode == ROW_NORMS;  // residual norms only (no z-update, no d, no spectrum)
  T tau = a.tau, mur = a.mu, dsc = T(1);
  if (a.mu_img) {
    const int img = (int)(Dp - a.desc);
    tau = T(a.lam64 / (norms ? a.mu_img[img] : a.mu_prev_img[img]));
    mur = T(a.mu_img[img]);
    dsc = T(a.dscale_img[img]);
  }
  const T tau2 = tau * tau, relax = a.relax;
  cx<T> *vb = reinterpret_cast<cx<T> *>(a.vbuf);
  // Statistics: per-thread partials in the working precision, only when
  // requested (the FP64 pipe is slow); FP64 for the CTA and plan reductions.
  const bool stats = a.partials != nullptr;
  T s_dd = T(0), s_dz = T(0), s_fit = T(0), s_tv = T(0), s_dv = T(0);
  for (int e = threadIdx.x; e < (nr + 1) * N; e += NT) {
    const int h = e / N, n = e - h * N, i = wrapi(r0 - 1 + h, M);
    const int n1 = (n + 1 == N) ? 0 : n + 1;
    T ah[C], av[C], dh0[C], dv0[C];
    T s = T(0), tv = T(0);
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      const int sg = ch * nh + h;
      const T x0 = bufr[2 * (n * ld + sg)], xr = bufr[2 * (n1 * ld + sg)], xd = bufr[2 * (n * ld + sg + 1)];
      const T gh = xr - x0, gv = xd - x0;
      cx<T> dold = (din && !inner) ? din[px0 + ch * P + (long long)i * N + n] : mk<T>(T(0), T(0));
      dh0[ch] = dold.x;
      dv0[ch] = dold.y;
      ah[ch] = gh + dold.x;
      av[ch] = gv + dold.y;
      s += ah[ch] * ah[ch] + av[ch] * av[ch];
      tv += gh * gh + gv * gv;
    }
    const T g = g_one ? T(1) : (s > tau2 ? T(1) - tau * rsqrt_t<T>(s) : T(0));
    G[h * N + n] = g;
    if (h >= 1) {
#pragma unroll
      for (int ch = 0; ch < C; ++ch) {
        const int sg = ch * nh + h;
        const long long o = px0 + ch * P + (long long)i * N + n;
        const T dnh = (T(1) - g) * ah[ch], dnv = (T(1) - g) * av[ch];
        if (norms) {
          const cx<T> vo = vb[o], vn = mk<T>(g * ah[ch], g * av[ch]);
          s_dd += (dnh - dh0[ch]) * (dnh - dh0[ch]) + (dnv - dv0[ch]) * (dnv - dv0[ch]);
          s_dv += (vn.x - vo.x) * (vn.x - vo.x) + (vn.y - vo.y) * (vn.y - vo.y);
          vb[o] = vn;
          continue;
        }
        if (!inner) dout[o] = mk<T>(dsc * dnh, dsc * dnv);
        if (g_one && vb) vb[o] = mk<T>(g * ah[ch], g * av[ch]);  // v^0 = D x^0
        if (stats) s_dd += (dnh - dh0[ch]) * (dnh - dh0[ch]) + (dnv - dv0[ch]) * (dnv - dv0[ch]);
        const T yo = a.yt[o];
        T yn = yo;
        if (!init) {
          const T t = bufr[2 * (n * ld + sg) + 1];
          if (!mask_bit(a.mask, mword + ch * mplane, (long long)i * N + n)) {
            yn = relax * t - (relax - T(1)) * yo;
            a.yt[o] = yn;
            if (stats) s_dz += (yn - yo) * (yn - yo);
          } else if (stats) {
            s_fit += (yo - t) * (yo - t);
          }
        }
        if (a.x_out) a.x_out[o] = bufr[2 * (n * ld + sg)];
        bufr[2 * (n * ld + sg) + 1] = yn;  // second slot now holds y~^{i+1}
      }
      if (stats) s_tv += sqrt(tv);
    }
  }
  if (norms) {  // uniform: the whole CTA leaves here
    double dd = double(s_dd), dv = double(s_dv), z = 0.0;
    block_sum3<NT>(dd, dv, z);
    if (threadIdx.x == 0) {
      a.apart[2 * (long long)(Dp->row_pbase + wi - Dp->row_begin)] = dd;
      a.apart[2 * (long long)(Dp->row_pbase + wi - Dp->row_begin) + 1] = dv;
    }
    return;
  }
  __syncthreads();

  // 3. r = mu D^T (v - d^{i+1}) with v - d^{i+1} = (2g - 1) a, on owned rows
  //    (((1+s) g - s) a and mu^{i+1} under penalty adaptation).
  T keep_y[KMAX * C], keep_r[KMAX * C];
  bool finite = true;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = threadIdx.x + k * NT;
    if (e < nr * N) {
      const int h = 1 + e / N, n = e - (h - 1) * N;
      const int i = r0 + h - 1, iu = wrapi(i - 1, M);
      const int nm = (n == 0) ? N - 1 : n - 1, n1 = (n + 1 == N) ? 0 : n + 1;
      const T s1 = T(1) + dsc;
      const T g0 = s1 * G[h * N + n] - dsc, gl = s1 * G[h * N + nm] - dsc, gu = s1 * G[(h - 1) * N + n] - dsc;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) {
        const int sg = ch * nh + h;
        const T x0 = bufr[2 * (n * ld + sg)], xl = bufr[2 * (nm * ld + sg)], xr = bufr[2 * (n1 * ld + sg)];
        const T xd = bufr[2 * (n * ld + sg + 1)], xu = bufr[2 * (n * ld + sg - 1)];
        const long long rowo = px0 + ch * P;
        const bool rd = din && !inner;
        cx<T> d0 = rd ? din[rowo + (long long)i * N + n] : mk<T>(T(0), T(0));
        cx<T> dl = rd ? din[rowo + (long long)i * N + nm] : mk<T>(T(0), T(0));
        cx<T> du = rd ? din[rowo + (long long)iu * N + n] : mk<T>(T(0), T(0));
        const T uh0 = g0 * (xr - x0 + d0.x), uhl = gl * (x0 - xl + dl.x);
        const T uv0 = g0 * (xd - x0 + d0.y), uvu = gu * (x0 - xu + du.y);
        const T r = inner ? T(0) : mur * ((uhl - uh0) + (uvu - uv0));
        const T yv = bufr[2 * (n * ld + sg) + 1];
        keep_y[k * C + ch] = yv;
        keep_r[k * C + ch] = r;
        finite = finite && isfinite(r) && isfinite(yv);
      }
    }
  }
  if (!finite) atomicOr(a.err, 1);
  __syncthreads();

  // 4. y~^{i+1} + i r into the compact forward layout (owned rows only).
  const int S2 = C * nr, ld2 = S2 | 1;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int e = threadIdx.x + k * NT;
    if (e < nr * N) {
      const int hh = e / N, n = e - hh * N;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) buf[n * ld2 + ch * nr + hh] = mk<T>(keep_y[k * C + ch], keep_r[k * C + ch]);
    }
  }
  __syncthreads();
  fft_smem<T, NT, -1>(buf, N, S2, ld2, sc, tw);

  // 5. Split the packed row spectrum C = Y + i R (Y, R Hermitian) and store.
  for (int e = threadIdx.x; e < nr * Nh; e += NT) {
    const int hh = e / Nh, k = e - hh * Nh, i = r0 + hh;
    const int km = (k == 0) ? 0 : N - k;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      const cx<T> c1 = buf[k * ld2 + ch * nr + hh], c2 = buf[km * ld2 + ch * nr + hh];
      cpair<T> q;
      q.ar = T(0.5) * (c1.x + c2.x);
      q.ai = T(0.5) * (c1.y - c2.y);
      q.br = T(0.5) * (c1.y + c2.y);
      q.bi = T(0.5) * (c2.x - c1.x);
      cpair<T> *dst = &a.S_out[spec0 + ((long long)ch * M + i) * Nh + k];
      if (inner)
        *reinterpret_cast<cx<T> *>(dst) = mk<T>(q.ar, q.ai);  // Y only; the R half is kept
      else
        st_pair(dst, q);
    }
  }

  if (stats) {
    double fit = 0.5 * double(s_fit) + double(a.lambda) * double(s_tv), dd = double(s_dd), dz = double(s_dz);
    block_sum3<NT>(dd, dz, fit);
    if (threadIdx.x == 0) {
      double *o = a.partials + 3 * (long long)(Dp->row_pbase + wi - Dp->row_begin);
      o[0] = dd;
      o[1] = dz;
      o[2] = fit;
    }
  }
}

// --------------------------------------------------------------- column ---
// Grid: one CTA per (image, channel, tile of W spectral columns k2).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) col_pass_kernel(ColArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wi = blockIdx.x;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, false)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh;
  const int local = wi - Dp->col_begin;
  const int ch = local / Dp->col_tiles, t = local - ch * Dp->col_tiles;
  const int k20 = t * Dp->W, w = min(Dp->W, Nh - k20);
  const int S = 2 * w, ld = S | 1;
  const FftSched sc = Dp->sched_col;
  const cx<T> *tw = reinterpret_cast<const cx<T> *>(a.tw) + Dp->tw_col;
  const cx<T> *H = reinterpret_cast<const cx<T> *>(a.hhat) + Dp->hhat;
  const T *s2c = a.s2 + Dp->s2_col, *s2r = a.s2 + Dp->s2_row;
  cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
  const long long base = Dp->spec + (long long)ch * M * Nh + k20;

  griddep_wait();
  for (int e = threadIdx.x; e < M * w; e += NT) {
    const int i = e / w, ww = e - i * w;
    const cpair<T> q = ld_pair(&a.S_in[base + (long long)i * Nh + ww]);
    buf[i * ld + 2 * ww] = mk<T>(q.ar, q.ai);
    buf[i * ld + 2 * ww + 1] = mk<T>(q.br, q.bi);
  }
  __syncthreads();
  fft_smem<T, NT, -1>(buf, M, S, ld, sc, tw);

  // Spectral solve of the x-step and the blur of its result.
  const T mu = a.mu_img ? T(a.mu_img[Dp - a.desc]) : a.mu, tikh = a.tikh, scale = T(1) / (T(M) * T(N));
  for (int e = threadIdx.x; e < M * w; e += NT) {
    const int k1 = e / w, ww = e - k1 * w, k2 = k20 + ww;
    const cx<T> h = __ldg(&H[(long long)k1 * Nh + k2]);
    const T den = h.x * h.x + h.y * h.y + (tikh > T(0) ? tikh : mu * (__ldg(&s2c[k1]) + __ldg(&s2r[k2])));
    const T inv = scale / den;
    const cx<T> Y = buf[k1 * ld + 2 * ww], R = tikh > T(0) ? mk<T>(T(0), T(0)) : buf[k1 * ld + 2 * ww + 1];
    const cx<T> X = cscale<T>(cadd<T>(cmulc<T>(h, Y), R), inv);
    buf[k1 * ld + 2 * ww] = X;
    buf[k1 * ld + 2 * ww + 1] = cmul<T>(h, X);
  }
  __syncthreads();
  fft_smem<T, NT, +1>(buf, M, S, ld, sc, tw);

  for (int e = threadIdx.x; e < M * w; e += NT) {
    const int i = e / w, ww = e - i * w;
    const cx<T> X = buf[i * ld + 2 * ww], HX = buf[i * ld + 2 * ww + 1];
    cpair<T> q;
    q.ar = X.x;
    q.ai = X.y;
    q.br = HX.x;
    q.bi = HX.y;
    st_pair(&a.S_out[base + (long long)i * Nh + ww], q);
  }
}

}  // namespace dcv
