// Row and column passes for power-of-two lengths L = 32 TT (64 .. 1024),
// built on the register-resident transform fft_p2 (fft.cuh).  Same
// arithmetic as the generic passes in iter_kernels.cuh (see the comment
// there for the iteration), different work decomposition:
//
//   row pass:    one group of TT threads per (channel, row) of the block,
//                rows r0-1 .. r1 (halo included); blockDim = C (Rb+2) TT.
//                Each thread owns the pixels q + TT m of its row, in
//                registers across the whole pass.
//   column pass: one group of TT threads per signal (Y or R of one spectral
//                column); the column tile is staged through shared memory
//                with coalesced row loads and stores.
#pragma once

#include "fft.cuh"
#include "internal.h"
#include "iter_kernels.cuh"

namespace dcv {

__device__ __forceinline__ unsigned group_mask(int TT) {
  if (TT >= 32) return 0xffffffffu;
  const int base = (threadIdx.x & 31) / TT * TT;
  return ((1u << TT) - 1u) << base;
}

// ------------------------------------------------------------------ row ---
template <typename T, int TT, int C>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) row_pass_p2_kernel(RowArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GS = p2_group_stride<TT>();
  const int wi = blockIdx.x;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, true)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh;
  const int blk = wi - Dp->row_begin;
  const int r0 = blk * Dp->Rb;
  const int nr = min(Dp->Rb, M - r0), nh = nr + 2;
  const long long P = (long long)M * N, px0 = Dp->px, spec0 = Dp->spec;
  const long long mword = Dp->mask, mplane = Dp->mask_plane;
  const cx<T> *tw2 = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->tw2_row;
  const cx<T> *din = reinterpret_cast<const cx<T> *>(a.d_in);
  cx<T> *dout = reinterpret_cast<cx<T> *>(a.d_out);
  const bool init = a.mode == ROW_INIT;

  const int g = threadIdx.x / TT, q = threadIdx.x - g * TT;
  const unsigned gm = group_mask(TT);
  const int ch = g / (Dp->Rb + 2), h = g - ch * (Dp->Rb + 2);  // this group's (channel, row)
  const bool active = ch < C && h < nh;
  const int i = wrapi(r0 - 1 + h, M);
  cx<T> *tile = reinterpret_cast<cx<T> *>(smem_raw) + (size_t)g * GS;
  // After the transforms, the same shared memory holds x, y~^{i+1} and g.
  T *X = reinterpret_cast<T *>(smem_raw);  // [C][nh][N]
  T *Yn = X + (size_t)C * nh * N;          // [C][nr][N]
  T *Gv = Yn + (size_t)C * nr * N;         // [nr+1][N]

  cx<T> v[32];
  // 1. x + i T~x on this group's row (inverse row DFT), or x^0 = y~0.
  if (active) {
    const long long rowp = px0 + ch * P + (long long)i * N;
    if (init) {
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = mk<T>(a.yt[rowp + q + TT * p2_slot<TT>(r)], T(0));
    } else {
      const cpair<T> *src = a.S_in + spec0 + ((long long)ch * M + i) * Nh;
#pragma unroll
      for (int m = 0; m < 32; ++m) {
        const int n = q + TT * m;
        if (2 * n <= N) {
          const cpair<T> c = src[n];
          v[m] = mk<T>(c.ar - c.bi, c.ai + c.br);
        } else {
          const cpair<T> c = src[N - n];
          v[m] = mk<T>(c.ar + c.bi, c.br - c.ai);
        }
      }
      fft_p2<T, TT, +1>(v, tile, q, gm, tw2);
    }
  }
  __syncthreads();

  // 2. x to shared memory; z-update on owned rows.
  const T relax = a.relax;
  double s_dd = 0.0, s_dz = 0.0, s_fit = 0.0, s_tv = 0.0;
  if (active) {
    const long long rowp = px0 + ch * P + (long long)i * N;
    const bool owned = h >= 1 && h <= nr;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int p = q + TT * p2_slot<TT>(r);
      X[((size_t)ch * nh + h) * N + p] = v[r].x;
      if (owned) {
        const T yo = a.yt[rowp + p];
        T yn = yo;
        if (!init) {
          if (!mask_bit(a.mask, mword + ch * mplane, (long long)i * N + p)) {
            yn = relax * v[r].y - (relax - T(1)) * yo;
            a.yt[rowp + p] = yn;
            s_dz += double(yn - yo) * double(yn - yo);
          } else {
            s_fit += double(yo - v[r].y) * double(yo - v[r].y);
          }
        }
        Yn[((size_t)ch * nr + h - 1) * N + p] = yn;
        if (a.x_out) a.x_out[rowp + p] = v[r].x;
      }
    }
  }
  __syncthreads();

  // 3. g = max(1 - tau/||a||, 0) on rows r0-1 .. r1-1 (one group per row,
  //    all channels), d^{i+1} = (1 - g) a on owned rows.
  const T tau = a.tau, tau2 = a.tau * a.tau;
  if (g <= nr) {
    const int hh = g, ii = wrapi(r0 - 1 + hh, M);
#pragma unroll 4
    for (int m = 0; m < 32; ++m) {
      const int p = q + TT * m, p1 = (p + 1 == N) ? 0 : p + 1;
      T ah[C], av[C], dh0[C], dv0[C];
      T s = T(0), tv = T(0);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T *Xr = X + ((size_t)c * nh + hh) * N;
        const T x0 = Xr[p], gh = Xr[p1] - x0, gv = Xr[N + p] - x0;
        const cx<T> dold = din ? din[px0 + c * P + (long long)ii * N + p] : mk<T>(T(0), T(0));
        dh0[c] = dold.x;
        dv0[c] = dold.y;
        ah[c] = gh + dold.x;
        av[c] = gv + dold.y;
        s += ah[c] * ah[c] + av[c] * av[c];
        tv += gh * gh + gv * gv;
      }
      const T gg = init ? T(1) : (s > tau2 ? T(1) - tau * rsqrt_t<T>(s) : T(0));
      Gv[(size_t)hh * N + p] = gg;
      if (hh >= 1) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const T dnh = (T(1) - gg) * ah[c], dnv = (T(1) - gg) * av[c];
          dout[px0 + c * P + (long long)ii * N + p] = mk<T>(dnh, dnv);
          s_dd += double(dnh - dh0[c]) * double(dnh - dh0[c]) + double(dnv - dv0[c]) * double(dnv - dv0[c]);
        }
        s_tv += sqrt(double(tv));
      }
    }
  }
  __syncthreads();

  // 4. r = mu D^T (v - d^{i+1}) on owned rows; v <- y~^{i+1} + i r.
  const bool fwd = active && h >= 1 && h <= nr;
  bool finite = true;
  if (fwd) {
    const T *Xr = X + ((size_t)ch * nh + h) * N;
    const T *Gr = Gv + (size_t)h * N;
    const long long dro = px0 + ch * P;
    const int iu = wrapi(i - 1, M);
#pragma unroll
    for (int m = 0; m < 32; ++m) {
      const int p = q + TT * m;
      const int pm = (p == 0) ? N - 1 : p - 1, p1 = (p + 1 == N) ? 0 : p + 1;
      const T x0 = Xr[p], xl = Xr[pm], xr = Xr[p1], xd = Xr[N + p], xu = Xr[p - N];
      const T g0 = T(2) * Gr[p] - T(1), gl = T(2) * Gr[pm] - T(1), gu = T(2) * Gr[p - N] - T(1);
      const cx<T> d0 = din ? din[dro + (long long)i * N + p] : mk<T>(T(0), T(0));
      const cx<T> dl = din ? din[dro + (long long)i * N + pm] : mk<T>(T(0), T(0));
      const cx<T> du = din ? din[dro + (long long)iu * N + p] : mk<T>(T(0), T(0));
      const T uh0 = g0 * (xr - x0 + d0.x), uhl = gl * (x0 - xl + dl.x);
      const T uv0 = g0 * (xd - x0 + d0.y), uvu = gu * (x0 - xu + du.y);
      const T r = a.mu * ((uhl - uh0) + (uvu - uv0));
      const T yv = Yn[((size_t)ch * nr + h - 1) * N + p];
      finite = finite && isfinite(r) && isfinite(yv);
      v[m] = mk<T>(yv, r);
    }
  }
  if (!finite) atomicOr(a.err, 1);
  __syncthreads();

  // 5. Forward row DFT of y~ + i r, then split C = Y + i R and store.
  if (fwd) {
    fft_p2<T, TT, -1>(v, tile, q, gm, tw2);
#pragma unroll
    for (int r = 0; r < 32; ++r) tile[q + TT * p2_slot<TT>(r)] = v[r];
    __syncwarp(gm);
    cpair<T> *dst = a.S_out + spec0 + ((long long)ch * M + i) * Nh;
    for (int k = q; k < Nh; k += TT) {
      const cx<T> c1 = tile[k], c2 = tile[k == 0 ? 0 : N - k];
      cpair<T> o;
      o.ar = T(0.5) * (c1.x + c2.x);
      o.ai = T(0.5) * (c1.y - c2.y);
      o.br = T(0.5) * (c1.y + c2.y);
      o.bi = T(0.5) * (c2.x - c1.x);
      dst[k] = o;
    }
  }

  if (a.partials) {
    double fit = 0.5 * s_fit + double(a.lambda) * s_tv;
    block_sum3_dyn(s_dd, s_dz, fit);
    if (threadIdx.x == 0) {
      double *o = a.partials + 3 * (long long)(Dp->row_pbase + blk);
      o[0] = s_dd;
      o[1] = s_dz;
      o[2] = fit;
    }
  }
}

// --------------------------------------------------------------- column ---
template <typename T, int TT>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) col_pass_p2_kernel(ColArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GS = p2_group_stride<TT>();
  const int wi = blockIdx.x;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, false)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh;
  const int local = wi - Dp->col_begin;
  const int ch = local / Dp->col_tiles, t = local - ch * Dp->col_tiles;
  const int k20 = t * Dp->W, w = min(Dp->W, Nh - k20);
  const int SL = (2 * Dp->W) | 1;  // staging row stride (complex)
  const cx<T> *tw2 = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->tw2_col;
  const cx<T> *H = reinterpret_cast<const cx<T> *>(a.hhat) + Dp->hhat;
  const T *s2c = a.s2 + Dp->s2_col, *s2r = a.s2 + Dp->s2_row;
  cx<T> *st = reinterpret_cast<cx<T> *>(smem_raw);  // [M][SL]
  const int g = threadIdx.x / TT, q = threadIdx.x - g * TT;
  const unsigned gm = group_mask(TT);
  cx<T> *tile = st + (size_t)M * SL + (size_t)g * GS;
  const long long base = Dp->spec + (long long)ch * M * Nh + k20;
  const int nthr = blockDim.x;

  for (int e = threadIdx.x; e < M * w; e += nthr) {
    const int ii = e / w, ww = e - ii * w;
    const cpair<T> c = a.S_in[base + (long long)ii * Nh + ww];
    st[ii * SL + 2 * ww] = mk<T>(c.ar, c.ai);
    st[ii * SL + 2 * ww + 1] = mk<T>(c.br, c.bi);
  }
  __syncthreads();
  cx<T> v[32];
  const bool active = g < 2 * w;
  if (active) {
#pragma unroll
    for (int m = 0; m < 32; ++m) v[m] = st[(q + TT * m) * SL + g];
    fft_p2<T, TT, -1>(v, tile, q, gm, tw2);
#pragma unroll
    for (int r = 0; r < 32; ++r) st[(q + TT * p2_slot<TT>(r)) * SL + g] = v[r];
  }
  __syncthreads();
  const T mu = a.mu, scale = T(1) / (T(M) * T(N));
  for (int e = threadIdx.x; e < M * w; e += nthr) {
    const int k1 = e / w, ww = e - k1 * w, k2 = k20 + ww;
    const cx<T> hv = __ldg(&H[(long long)k1 * Nh + k2]);
    const T den = hv.x * hv.x + hv.y * hv.y + mu * (__ldg(&s2c[k1]) + __ldg(&s2r[k2]));
    const T inv = scale / den;
    const cx<T> Y = st[k1 * SL + 2 * ww], R = st[k1 * SL + 2 * ww + 1];
    const cx<T> Xv = cscale<T>(cadd<T>(cmulc<T>(hv, Y), R), inv);
    st[k1 * SL + 2 * ww] = Xv;
    st[k1 * SL + 2 * ww + 1] = cmul<T>(hv, Xv);
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int m = 0; m < 32; ++m) v[m] = st[(q + TT * m) * SL + g];
    fft_p2<T, TT, +1>(v, tile, q, gm, tw2);
#pragma unroll
    for (int r = 0; r < 32; ++r) st[(q + TT * p2_slot<TT>(r)) * SL + g] = v[r];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < M * w; e += nthr) {
    const int ii = e / w, ww = e - ii * w;
    const cx<T> Xv = st[ii * SL + 2 * ww], HX = st[ii * SL + 2 * ww + 1];
    cpair<T> c;
    c.ar = Xv.x;
    c.ai = Xv.y;
    c.br = HX.x;
    c.bi = HX.y;
    a.S_out[base + (long long)ii * Nh + ww] = c;
  }
}

}  // namespace dcv
