// Fused row pass of one plain iteration (one block-Gauss-Seidel pass, fixed
// penalty, no statistics): the inverse half and the forward half of
// iter_p2.cuh in one kernel, so that x is not written by one launch and read
// back by the next, and y~ is read once.
//
// The forward half of row f needs x on rows f-1, f, f+1 and the updated y~
// of row f.  A work item owns rows [r0, r0 + nr) of an image: it runs the
// inverse half (x, T~x, z-update) of those rows, publishes them, and then
// runs the forward half of rows [r0 - 1, r0 + nr - 1), shifted down by one
// row, so that it needs x only from its own rows and from items of lower
// index of the same image (rows r0 - 2, r0 - 1).  The periodic boundary
// closes the chain: the image's first item also computes x of row M - 1
// (into a per-image halo row, without the z-update) and runs the forward
// half of its rows [0, nr - 1); the last item also runs the forward half of
// row M - 1 (x of row 0 comes from the first item).
//
// Items are taken in order from a per-class ticket counter (ticket mod
// items = item, ticket / items + 1 = the launch's epoch), and an item waits
// only for flags of items with smaller tickets of the same launch.  Those
// were taken by CTAs that are already running and that never wait on a
// larger ticket, so every wait ends; each wait is also bounded by a
// globaltimer limit, after which the item sets bit 2 of the error word
// (DECONV_ETIMEOUT on the host), skips its forward half and returns.
#pragma once

#include "iter_p2.cuh"

namespace dcv {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until *f has reached epoch (modulo 2^32); false when limit_ns
// nanoseconds passed first.  The clock is read before the flag, so a limit
// of 0 never waits (and always fails).
__device__ __forceinline__ bool wait_flag(const unsigned *f, unsigned epoch, long long limit_ns) {
  const unsigned long long t0 = global_ns();
  unsigned sleep_ns = 32;
  for (;;) {
    if ((long long)(global_ns() - t0) >= limit_ns) return false;
    if ((int)(ld_acquire_u32(f) - epoch) >= 0) return true;
    __nanosleep(sleep_ns);
    if (sleep_ns < 1024) sleep_ns *= 2;
  }
}

// Register cap: three-channel FP32 rows with 16 values per thread, 72 for
// R = 3, 5 (three 288-thread CTAs per SM; measured faster than 80 despite
// the spills of holding both halves' live ranges) and 96 for R = 1.
template <typename T, int C, int R, int V> __host__ __device__ constexpr int fused_reg_cap() {
  return (C == 3 && V == 16 && sizeof(T) == 4) ? (R == 1 ? 96 : 72) : (sizeof(T) == 4 ? 128 : 255);
}

// Same CTA layout as the two halves: R groups of TT threads per (channel,
// row slot), Rb row slots.  Shared memory: the inverse half's (one region of
// R transpose tiles per (channel, row slot), y~ rows, mask words); the
// forward half reuses the regions.
template <typename T, int TT, int C, int R, int V>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) __maxnreg__((fused_reg_cap<T, C, R, V>()))
    row_fused_p2_kernel(RowArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GS = reg_group_stride<V, TT>(), L2 = V * TT, RS = R * GS;
  static_assert((R * V * TT) % 32 == 0, "the pixel-major step takes whole 32-pixel runs of a row");
  __shared__ unsigned long long s_ticket;
  __shared__ int s_ok;
  griddep_wait();
  if (threadIdx.x == 0) s_ticket = atomicAdd(a.ticket, 1ULL);
  __syncthreads();
  const unsigned long long tk = s_ticket;
  const int wi = (int)(tk % (unsigned long long)a.items);
  const unsigned epoch = (unsigned)(tk / (unsigned long long)a.items) + 1u;
  const ImageDesc *Dp = &a.desc[find_item(a.desc, a.cls_imgs, a.nimg, wi, true)];
  const int M = Dp->M, N = Dp->N, Nh = Dp->Nh, Rb = Dp->Rb, wpr = N / 32;
  const int blk = wi - Dp->row_begin;
  const int r0 = blk * Rb, nr = min(Rb, M - r0);
  const bool first = blk == 0, last = blk == Dp->row_blocks - 1;
  const bool halo = first && !last;  // this item computes x of row M - 1 for the image's other items
  const long long P = (long long)M * N, px0 = Dp->px;
  const int g = threadIdx.x / TT, q = threadIdx.x - g * TT;
  const int bar = 1 + g;  // named barrier of a 64-thread group (group_bar)
  const int gr = g % R, row_id = g / R, ch = row_id / Rb, hh = row_id - ch * Rb;
  const unsigned gm = group_mask(TT);
  cx<T> *Reg = reinterpret_cast<cx<T> *>(smem_raw) + (size_t)row_id * RS;  // this slot's region
  cx<T> *tile = Reg + gr * GS;
  T *Ys = reinterpret_cast<T *>(reinterpret_cast<cx<T> *>(smem_raw) + (size_t)C * Rb * RS);  // [C][Rb][N]
  uint32_t *Ms = reinterpret_cast<uint32_t *>(Ys + (size_t)C * Rb * N);              // [C][Rb][N/32]
  const cx<T> *tw2 = reinterpret_cast<const cx<T> *>(a.tw2) + (V == 32 ? Dp->tw2_row : Dp->tw16_row);
  const cx<T> *tw3 = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->tw3_row;
  const cx<T> *twab = reinterpret_cast<const cx<T> *>(a.tw2) + Dp->twab_row;
  T *yt = a.yt;
  T *xbuf = a.xbuf;
  T *hrow = a.halo + Dp->halo;  // [C][N]: x of row M - 1, computed by the first item
  T *xout = (a.x_out && a.x_out != a.xbuf) ? a.x_out : nullptr;
  bool finite = true;

  // ---- inverse half: own rows (z-update), then the halo row -------------
  for (int c = 0; c < C; ++c) {
    copy_async<T>(Ys + (size_t)c * Rb * N, yt + px0 + c * P + (long long)r0 * N, nr * N, threadIdx.x, blockDim.x);
    copy_async<uint32_t>(Ms + (size_t)c * Rb * wpr, a.mask + Dp->mask + c * Dp->mask_plane + (long long)r0 * wpr,
                         nr * wpr, threadIdx.x, blockDim.x);
  }
  cp_async_commit();
  const int ninv = nr + (halo ? 1 : 0), inv_rounds = (ninv + Rb - 1) / Rb;
  for (int rd = 0; rd < inv_rounds; ++rd) {
    const int j = rd * Rb + hh;
    const bool own = j < nr, is_halo = halo && j == nr;
    const bool active = ch < C && (own || is_halo);
    const int i = own ? r0 + j : M - 1;
    cx<T> v[V];
    if (active) {
      const cpair<T> *src = a.S_in + Dp->spec + ((long long)ch * M + i) * Nh;
#pragma unroll
      for (int m = 0; m < V; ++m) {
        const int n = R * (q + TT * m) + gr;
        const cpair<T> c = src[2 * n <= N ? n : N - n];
        v[m] = 2 * n <= N ? mk<T>(c.ar - c.bi, c.ai + c.br) : mk<T>(c.ar + c.bi, c.br - c.ai);
      }
    }
    fft_reg<T, V, TT, R, +1>(v, active, tile, q, gm, bar, gr, tw2, tw3, twab, Reg);
    if (rd == 0) cp_async_wait_all();
    __syncthreads();
    if (active && own) {
      const long long rowp = px0 + ch * P + (long long)i * N;
      const T relax = a.relax;
      const T *yrow = Ys + ((size_t)ch * Rb + j) * N;
      const uint32_t *mrow = Ms + ((size_t)ch * Rb + j) * wpr;
#pragma unroll
      for (int jj = 0; jj < V; ++jj) {
        const int p = reg_pos<V, TT>(q, jj) + L2 * gr;
        xbuf[rowp + p] = v[jj].x;
        if (xout) xout[rowp + p] = v[jj].x;
        if (!((mrow[p >> 5] >> (p & 31)) & 1u)) yt[rowp + p] = relax * v[jj].y - (relax - T(1)) * yrow[p];
      }
    } else if (active) {
#pragma unroll
      for (int jj = 0; jj < V; ++jj) {
        const int p = reg_pos<V, TT>(q, jj) + L2 * gr;
        hrow[ch * N + p] = v[jj].x;
      }
    }
    __syncthreads();  // the regions are reused; every write is done before the publication
  }

  // ---- publish, then wait for the items this one reads from -------------
  if (threadIdx.x == 0) {
    __threadfence();
    st_release_u32(&a.flags[wi], epoch);
    bool ok = true;
    if (!first) {
      ok = wait_flag(&a.flags[wi - 1], epoch, a.wait_ns);
      if (ok && Rb == 1 && blk >= 2) ok = wait_flag(&a.flags[wi - 2], epoch, a.wait_ns);
      if (ok && last) ok = wait_flag(&a.flags[wi - blk], epoch, a.wait_ns);
    }
    if (!ok) atomicOr(a.err, 2);
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  if (!s_ok) return;  // uniform: the whole CTA leaves (its forward rows stay stale; the host reports the timeout)

  // ---- forward half of rows [fbeg, fend) --------------------------------
  const int fbeg = first ? 0 : r0 - 1, fend = last ? M : r0 + nr - 1;
  const int fwd_rounds = (fend - fbeg + Rb - 1) / Rb;
  const T tau = a.tau, tau2 = tau * tau, mu = a.mu;
  const cx<T> *dg = reinterpret_cast<const cx<T> *>(a.d_in) + px0;
  cx<T> *dout = reinterpret_cast<cx<T> *>(a.d_out);
  // x of a row of channel c: the halo copy of row M - 1 for every item but
  // the last (which owns that row), the x buffer otherwise.
  auto xrow = [&](int c, int row) -> const T * {
    return (row == M - 1 && !last) ? hrow + c * N : xbuf + px0 + c * P + (long long)row * N;
  };
  for (int rd = 0; rd < fwd_rounds; ++rd) {
    const int f = fbeg + rd * Rb + hh;
    const bool active = ch < C && f < fend;
    const int fu = f == 0 ? M - 1 : f - 1, fd = f + 1 == M ? 0 : f + 1;
    if (a.prefetch)
      prefetch_fwd_rows<T, C>(xrow, dg, yt + px0, P, M, N, fbeg + rd * Rb, min(Rb, fend - (fbeg + rd * Rb)), false);
    cx<T> v[V];
    if constexpr (C > 1) {
      // the pixel-major prox step (norm over channels in the thread)
      const int f0 = fbeg + rd * Rb;
      T no_dd = T(0), no_tv = T(0);
      finite = prox_rows_pm<T, C>(xrow, dg, yt + px0, dout + px0, P, M, N, f0, min(Rb, fend - f0), false, tau, mu,
                                  reinterpret_cast<cx<T> *>(smem_raw), (size_t)Rb * RS, (size_t)RS, false, no_dd,
                                  no_tv) &&
               finite;
      __syncthreads();  // the rows' y~ + i r are in the regions
      if (active) {
#pragma unroll
        for (int m = 0; m < V; ++m) v[m] = Reg[R * (q + TT * m) + gr];
      }
      // every group of the row has read its inputs before the tiles overwrite them
      if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
    } else {
      if (active) {
        const T *xr = xrow(0, f), *xu = xrow(0, fu), *xd = xrow(0, fd);
        const cx<T> *dr = dg + (long long)f * N, *dru = dg + (long long)fu * N;
        const T *yrow = yt + px0 + (long long)f * N;
#pragma unroll 4
        for (int m = 0; m < V; ++m) {
          const int p = q + TT * m + L2 * gr;
          const int pm = (p == 0) ? N - 1 : p - 1, p1 = (p + 1 == N) ? 0 : p + 1;
          const T x0 = xr[p], xl = xr[pm], xrr = xr[p1], xdn = xd[p], xdl = xd[pm], xup = xu[p], xul = xu[p1];
          const cx<T> d0 = dr[p], dl = dr[pm], du = dru[p];
          const T ah0 = (xrr - x0) + d0.x, av0 = (xdn - x0) + d0.y;
          const T ahl = (x0 - xl) + dl.x, avl = (xdl - xl) + dl.y;
          const T ahu = (xul - xup) + du.x, avu = (x0 - xup) + du.y;
          const T s0 = sq2<T>(ah0, av0), sl = sq2<T>(ahl, avl), su = sq2<T>(ahu, avu);
          const T g0 = shrink_g<T>(s0, tau, tau2), gl = shrink_g<T>(sl, tau, tau2), gu = shrink_g<T>(su, tau, tau2);
          dout[px0 + (long long)f * N + p] = mk<T>(prox_d<T>(g0, ah0), prox_d<T>(g0, av0));
          const T r = prox_r<T>(mu, gl, ahl, g0, ah0, gu, avu, av0);
          const T yv = yrow[p];
          finite = finite && isfinite(r) && isfinite(yv);
          Reg[p] = mk<T>(yv, r);
        }
      }
      if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
      if (active) {
#pragma unroll
        for (int m = 0; m < V; ++m) v[m] = Reg[R * (q + TT * m) + gr];
      }
      // every group of the row has read its inputs before the tiles overwrite them
      if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
    }
    fft_reg_smem<T, V, TT, R, -1>(v, active, tile, q, gm, bar, gr, tw2, tw3, twab, Reg);
    if (R > 1) __syncthreads(); else group_bar<TT>(gm, bar);
    if (active) {
      cpair<T> *dst = a.S_out + Dp->spec + ((long long)ch * M + f) * Nh;
      for (int k = q + TT * gr; k < Nh; k += TT * R) {
        const cx<T> c1 = Reg[k], c2 = Reg[k == 0 ? 0 : N - k];
        cpair<T> o;
        o.ar = T(0.5) * (c1.x + c2.x);
        o.ai = T(0.5) * (c1.y - c2.y);
        o.br = T(0.5) * (c1.y + c2.y);
        o.bi = T(0.5) * (c2.x - c1.x);
        dst[k] = o;
      }
    }
    __syncthreads();  // the next round's inputs overwrite the regions
  }
  if (!finite) atomicOr(a.err, 1);
}

}  // namespace dcv
