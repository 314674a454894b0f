// Host side of the C ABI declared in include/deconv.h: argument validation,
// workspace layout, plan setup (H^, packed masks, twiddle tables) and the
// iteration driver (direct launches, or a cached CUDA graph of a fixed number
// of iterations replayed on the caller's stream).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "deconv.h"
#include "internal.h"

using namespace dcv;

namespace {

constexpr int kGraphIters = 20;          // iterations per captured graph (even: d ping-pong returns to 0)
constexpr int kTargetCtas = 2 * 152;     // aim for two CTAs per SM on a 152-SM GB300
constexpr size_t kL2PrefetchMin = (size_t)64 << 20;  // workspace above which the forward half prefetches its rows
constexpr size_t kMaxSmem = 227 * 1024 - 2048;  // opt-in dynamic shared memory per CTA, minus static use
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool factor235(int L, FftSched *sc) {
  if (L < 1) return false;
  int a = 0, b = 0, c = 0, v = L;
  while (v % 2 == 0) { v /= 2; ++a; }
  while (v % 3 == 0) { v /= 3; ++b; }
  while (v % 5 == 0) { v /= 5; ++c; }
  if (v != 1) return false;
  sc->n16 = (int8_t)(a / 4);
  sc->r = (int8_t)(1 << (a % 4));
  sc->n5 = (int8_t)c;
  sc->n3 = (int8_t)b;
  return true;
}

constexpr int kDefaultGroupMiB = -1;      // image groups of the captured loop by default: none (one group)

// One kernel class of a pass: the images of one image group launched
// together with one kernel.
struct Cls {
  LaunchCfg cfg;
  int group = 0;
  std::vector<int> imgs;
  size_t o_imgs = 0;  // workspace offset of the image list
  size_t o_ticket = 0, o_flags = 0;  // fused row pass: ticket counter, one flag per work item
};

struct Layout {
  int B = 0, C = 0, K = 0, dtype = 0, nt = 256, kernel_per_image = 0;
  std::vector<Cls> row_cls, col_cls;
  // Image groups of the captured loop: the row and column classes of each;
  // chains: the groups run side by side (else one after another).
  int ngroups = 1;
  bool chains = false;
  std::vector<std::vector<int>> grp_row, grp_col;
  std::map<int, int> tw2_off;
  long long total_tw2 = 0;
  int total_row_items = 0;
  size_t esz = 4;
  std::vector<ImageDesc> desc;
  long long total_px = 0, total_spec = 0, total_hhat = 0, total_words = 0, total_tw = 0, total_s2 = 0;
  long long total_halo = 0;
  std::vector<HhatJob> jobs;
  std::vector<long long> job_begin, g_begin, img_word_begin, img_px_begin;
  long long total_g = 0;  // K x Nh row sums of every H^ job (double2)
  std::vector<int> plane_img;
  std::vector<int> lengths;
  std::map<int, int> tw_off, s2_off;
  long long hhat_total_elems = 0;
  int row_grid = 0, col_grid = 0;
  size_t row_smem = 0, col_smem = 0;
  size_t o_yt, o_d0, o_d1, o_Sa, o_Sb, o_hhat, o_bits, o_tw, o_tw2, o_s2, o_desc, o_jobs, o_jobbeg, o_wordbeg,
      o_pxbeg, o_planeimg, o_meanpart, o_means, o_partials, o_err, o_xbuf, o_clsimgs, o_v, o_mu, o_apart, o_halo,
      o_hg, o_gbeg,
      o_sync, sync_bytes, total;
};

bool is_pow2_32(int L) { return L >= 64 && L <= 1024 && (L & (L - 1)) == 0; }

// Register-FFT parameters of a length: L = r * 32 * tt with (tt, r) = (L/32, 1)
// for powers of two 64..1024, or r in {3, 5} and 32 * tt in {128, 256, 512}.
bool reg_fft_params(int L, int *tt, int *r, int *v = nullptr, int vpref = 32) {
  if (v) *v = 32;
  if (is_pow2_32(L)) {
    if (v && vpref == 16) {  // 16 values per thread: L / 16 threads (4..64)
      *v = 16;
      *tt = L / 16;
      *r = 1;
      return true;
    }
    *tt = L / 32;
    *r = 1;
    return true;
  }
  for (int rr : {3, 5})
    if (L % rr == 0) {
      const int L2 = L / rr;
      if (L2 >= 128 && L2 <= 512 && (L2 & (L2 - 1)) == 0) {
        if (v && vpref == 16) {
          *v = 16;
          *tt = L2 / 16;
        } else {
          *tt = L2 / 32;
        }
        *r = rr;
        return true;
      }
    }
  return false;
}

// Register-FFT kernel class key: values per thread, threads per sub-transform, radix.
int p2_key(int v, int tt, int r) { return (v == 16 ? 1000 : 0) + tt * 8 + r; }
void p2_unkey(int key, int *v, int *tt, int *r) {
  *v = key >= 1000 ? 16 : 32;
  *tt = (key % 1000) / 8;
  *r = key % 8;
}
int p2_group_stride_hv(int tt, int v) { return v == 16 ? v16_group_stride_h(tt) : p2_group_stride_h(tt); }

// Register-FFT row passes (inverse and forward halves): rb rows per CTA, r
// groups of tt threads per (channel, row), rounded up to whole warps.
int p2_row_threads(int C, int rb, int tt, int r = 1) {
  if (tt >= 32) return C * rb * r * tt;
  const int per_warp = 32 / tt;
  return (C * rb * r + per_warp - 1) / per_warp * per_warp * tt;
}

// Shared memory of one half of a register-FFT row pass (0: inverse, 1: forward).
size_t p2_row_smem_half(int C, int N, int rb, int tt, size_t esz, int r, int stage, int half, int v = 32) {
  const size_t gs = (size_t)p2_group_stride_hv(tt, v);
  const size_t region = (size_t)C * rb * r * gs * 2 * esz;  // tiles / exchange per row
  if (half == 0) return region + (size_t)C * rb * N * esz + (size_t)C * rb * (N / 32) * 4;  // + y~ rows, mask
  if (!stage) return region;
  // staged forward half: [x (rb+2) rows][d (rb+1) rows][y~ rb rows] (the tiles
  // reuse them), then y~ + i r and the exchange buffer per row
  const size_t tiles = (size_t)(p2_row_threads(C, rb, tt, r) / tt) * gs * 2 * esz;
  const size_t ex = r > 1 ? (size_t)C * rb * N * 2 * esz : 0;
  return std::max((size_t)C * ((rb + 2) + 2 * (rb + 1) + rb) * N * esz, tiles) + (size_t)C * rb * N * 2 * esz + ex;
}

size_t p2_row_smem(int C, int N, int rb, int tt, size_t esz, int r = 1, int stage = 0, int v = 32) {
  return std::max(p2_row_smem_half(C, N, rb, tt, esz, r, stage, 0, v),
                  p2_row_smem_half(C, N, rb, tt, esz, r, stage, 1, v));
}

// Column pass: one column of r transpose tiles (+4 padding) per signal, H^ tile, sin^2 tables.
size_t p2_col_smem(int M, int w, int tt, size_t esz, int r = 1, int v = 32) {
  return (size_t)2 * w * (r * p2_group_stride_hv(tt, v) + 4) * 2 * esz + (size_t)M * w * 2 * esz +
         (size_t)((M + w + 3) & ~3) * esz;
}

int p2_col_threads(int w, int tt, int r = 1) {
  if (tt >= 32) return 2 * w * r * tt;
  const int per_warp = 32 / tt;
  return (2 * w * r + per_warp - 1) / per_warp * per_warp * tt;
}

// Groups of 64 threads synchronise on named barriers 1..15: at most 15 per CTA.
bool p2_groups_ok(int threads, int tt) { return tt < 64 || threads / tt <= 15; }

// Row-block height and column-tile width for one image under CTA size nt.
bool fit_image(int M, int N, int C, int nt, size_t esz, int rb_pref, int w_pref, int *Rb, int *W) {
  const int budget = 30 * nt, kmax = 16 / C;
  int rb = std::min(budget / (C * N) - 2, kmax * nt / N);
  if (rb < 1) return false;
  rb = std::min(rb, std::max(1, rb_pref));
  rb = std::min(rb, M);
  while (rb >= 1) {
    size_t ld = (size_t)((C * (rb + 2)) | 1);
    size_t smem = (size_t)N * ld * 2 * esz + (size_t)(rb + 1) * N * esz;
    if (smem <= kMaxSmem) break;
    --rb;
  }
  if (rb < 1) return false;
  const int Nh = N / 2 + 1;
  int w = std::min(16, budget / (2 * M));
  if (w < 1) return false;
  w = std::min(w, std::max(1, w_pref));
  w = std::min(w, Nh);
  while (w >= 1 && (size_t)M * (size_t)((2 * w) | 1) * 2 * esz > kMaxSmem) --w;
  if (w < 1) return false;
  *Rb = rb;
  *W = w;
  return true;
}

// Tuning of the register-FFT passes (deconv_tune); NULL or entries <= 0 /
// < 0: the defaults (152 CTAs per row class and per column pass; the forward
// row half staged for one-channel single-class plans).
deconv_status build_layout(const deconv_dims *d, Layout *Lo, const deconv_tune *tune = nullptr) {
  if (!d || d->batch < 1 || !d->rows || !d->cols) return DECONV_EINVAL;
  if (d->channels != 1 && d->channels != 3) return DECONV_EINVAL;
  if (d->ksize < 1 || d->ksize % 2 == 0) return DECONV_EINVAL;
  if (d->dtype != DECONV_F32 && d->dtype != DECONV_F64) return DECONV_EINVAL;
  if (!(d->relax >= 1.0f && d->relax <= 2.0f)) return DECONV_EINVAL;
  if (d->kernel_per_image != 0 && d->kernel_per_image != 1) return DECONV_EINVAL;
  if (d->ksizes) {
    if (!d->kernel_per_image) return DECONV_EINVAL;
    for (int j = 0; j < d->batch; ++j)
      if (d->ksizes[j] < 1 || d->ksizes[j] % 2 == 0 || d->ksizes[j] > d->ksize) return DECONV_EINVAL;
  }
  Layout &L = *Lo;
  L.B = d->batch;
  L.C = d->channels;
  L.K = d->ksize;
  L.dtype = d->dtype;
  L.kernel_per_image = d->kernel_per_image;
  L.esz = d->dtype == DECONV_F32 ? 4 : 8;
  long long rows_total = 0, cols_total = 0;
  for (int j = 0; j < L.B; ++j) {
    const int M = d->rows[j], N = d->cols[j];
    if (M < d->ksize || N < d->ksize || M < 2 || N < 2) return DECONV_EINVAL;
    if ((long long)M * N > (1LL << 30)) return DECONV_EUNSUPPORTED;
    FftSched s;
    if (!factor235(M, &s) || !factor235(N, &s)) return DECONV_EUNSUPPORTED;
    rows_total += M;
    cols_total += (long long)L.C * (N / 2 + 1);
  }
  const int maxthr = L.esz == 4 ? 512 : 256;
  const bool allow_p2 = !(tune && tune->generic);
  // Kernel class of every image and pass: the register-FFT passes for the
  // lengths reg_fft_params accepts (key tt * 8 + r), the generic Stockham
  // passes otherwise (key 0).
  // Kernel key of every image and pass: the register-FFT class (key
  // p2_key(v, tt, r)) where reg_fft_params accepts the length, 0 = generic.
  std::vector<int> row_key(L.B, 0), col_key(L.B, 0);
  // Values per thread of the power-of-two register transforms: 16 (twice the
  // threads, so twice the resident warps) unless the tuning asks for 32.
  // Defaults (measured on GB300): rows 16; columns 32 for power-of-two
  // lengths, 16 for 3 * 2^k and 5 * 2^k.
  const int vrow = (tune && tune->fft_values > 0) ? tune->fft_values : 16;
  const int vcol_set = (tune && tune->col_fft_values > 0) ? tune->col_fft_values : 0;
  for (int j = 0; j < L.B; ++j) {
    const int M = d->rows[j], N = d->cols[j];
    int tt, r, v;
    if (allow_p2 && reg_fft_params(N, &tt, &r, &v, vrow) && p2_row_threads(L.C, 1, tt, r) <= maxthr &&
        p2_groups_ok(p2_row_threads(L.C, 1, tt, r), tt) && p2_row_smem(L.C, N, 1, tt, L.esz, r, L.C == 1, v) <= kMaxSmem)
      row_key[j] = p2_key(v, tt, r);
    const int vcol = vcol_set ? vcol_set : (is_pow2_32(M) ? 32 : 16);
    if (allow_p2 && reg_fft_params(M, &tt, &r, &v, vcol) && p2_col_threads(1, tt, r) <= maxthr &&
        p2_col_smem(M, 1, tt, L.esz, r, v) <= kMaxSmem)
      col_key[j] = p2_key(v, tt, r);
  }
  // Image groups of the captured loop.  Chains: one group per (row kernel,
  // column kernel) pair, the groups' iterations running side by side on
  // streams of their own.  Otherwise groups for L2 residency (first fit,
  // largest intermediate first): each group's row-spectral intermediate
  // within the budget, all iterations of one group before the next.
  std::vector<int> grp(L.B, 0);
  if (tune && tune->chains) {
    std::map<std::pair<int, int>, int> pair_grp;
    for (int j = 0; j < L.B; ++j) {
      auto it = pair_grp.find({row_key[j], col_key[j]});
      if (it == pair_grp.end()) it = pair_grp.emplace(std::make_pair(row_key[j], col_key[j]), (int)pair_grp.size()).first;
      grp[j] = it->second;
    }
    L.ngroups = (int)pair_grp.size();
    L.chains = L.ngroups > 1;
  } else {
    const int mb = (tune && tune->l2_group_mb != 0) ? tune->l2_group_mb : kDefaultGroupMiB;
    if (mb > 0) {
      const long long budget = (long long)mb << 20;
      std::vector<int> order(L.B);
      std::vector<long long> sb(L.B);
      for (int j = 0; j < L.B; ++j) {
        order[j] = j;
        sb[j] = (long long)L.C * d->rows[j] * (d->cols[j] / 2 + 1) * 4 * (long long)L.esz;
      }
      std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return sb[u] > sb[v]; });
      std::vector<long long> used;
      for (int j : order) {
        size_t g = 0;
        while (g < used.size() && used[g] + sb[j] > budget) ++g;
        if (g == used.size()) used.push_back(0);
        used[g] += sb[j];
        grp[j] = (int)g;
      }
      L.ngroups = (int)used.size();
    }
  }
  // Per-(group, kernel) keys: the kernel key plus the group times kGroupKey.
  constexpr int kGroupKey = 4096;
  long long g_rows = 0, g_cols = 0;
  std::map<int, long long> p2_rows, p2_cols;
  std::map<int, int> p2_row_keys;  // distinct register row kernels (any group)
  for (int j = 0; j < L.B; ++j) {
    const int M = d->rows[j], N = d->cols[j];
    if (row_key[j]) {
      p2_rows[grp[j] * kGroupKey + row_key[j]] += M;
      p2_row_keys[row_key[j]] = 1;
    } else {
      g_rows += M;
    }
    if (col_key[j])
      p2_cols[grp[j] * kGroupKey + col_key[j]] += (long long)L.C * (N / 2 + 1);
    else
      g_cols += (long long)L.C * (N / 2 + 1);
  }
  const int target = kTargetCtas;
  const int rb_pref = (int)std::max<long long>(2, (g_rows + target - 1) / target);
  const int w_pref = (int)std::max<long long>(1, (g_cols + target - 1) / target);
  // Generic CTA size: 256 threads when every generic image fits, else 512 (FP32 only).
  bool ok = false;
  for (int nt : {256, 512}) {
    if (nt != 256 && !(nt == 512 && L.esz == 4)) continue;
    bool all = true;
    for (int j = 0; j < L.B && all; ++j) {
      if (row_key[j] && col_key[j]) continue;
      int rb, w;
      all = fit_image(d->rows[j], d->cols[j], L.C, nt, L.esz, rb_pref, w_pref, &rb, &w);
    }
    if (all) {
      L.nt = nt;
      ok = true;
      break;
    }
  }
  if (!ok) return DECONV_EUNSUPPORTED;
  // Class parameters: rows per CTA / columns per CTA aiming at one CTA per SM.
  std::map<int, int> p2_rb, p2_w;
  // One channel and one row kernel: the forward row half stages its rows (x
  // with halo, d, y~) in shared memory.  Otherwise it reads them through L1:
  // the staged rows of three channels would leave room for one row per CTA,
  // and the classes of a batch run concurrently only while their CTAs fit on
  // the SMs side by side.
  int row_stage = (L.C == 1 && p2_row_keys.size() == 1 && g_rows == 0) ? 1 : 0;
  if (tune && tune->row_stage >= 0) row_stage = L.C == 1 ? (tune->row_stage ? 1 : 0) : 0;
  for (const auto &kv : p2_rows) {
    int v, tt, r;
    p2_unkey(kv.first % kGroupKey, &v, &tt, &r);
    const int N = r * v * tt;
    const int rtarget = (tune && tune->row_ctas > 0) ? tune->row_ctas : 152;
    int rb = (int)std::max<long long>(1, (kv.second + rtarget - 1) / rtarget);
    while (rb > 1 && (p2_row_threads(L.C, rb, tt, r) > maxthr || !p2_groups_ok(p2_row_threads(L.C, rb, tt, r), tt) ||
                      p2_row_smem(L.C, N, rb, tt, L.esz, r, row_stage, v) > kMaxSmem))
      --rb;
    p2_rb[kv.first] = rb;
  }
  std::vector<int> p2w_all(L.ngroups, 1);
  {
    std::vector<long long> tot(L.ngroups, 0);
    for (const auto &kv : p2_cols) tot[kv.first / kGroupKey] += kv.second;
    const int ctarget = (tune && tune->col_ctas > 0) ? tune->col_ctas : 152;
    for (int g = 0; g < L.ngroups; ++g) p2w_all[g] = (int)std::max<long long>(1, (tot[g] + ctarget - 1) / ctarget);
  }
  for (const auto &kv : p2_cols) {
    int v, tt, r;
    p2_unkey(kv.first % kGroupKey, &v, &tt, &r);
    const int M = r * v * tt;
    int w = std::min(p2w_all[kv.first / kGroupKey], 16);
    while (w > 1 && (p2_col_threads(w, tt, r) > maxthr || !p2_groups_ok(p2_col_threads(w, tt, r), tt) ||
                     p2_col_smem(M, w, tt, L.esz, r, v) > kMaxSmem))
      --w;
    p2_w[kv.first] = w;
  }

  // Class lists (in order of first appearance).
  auto class_index = [](std::vector<Cls> &v, int kind, int key, int group) {
    int vv = 32, tt = 0, r = 0;
    if (kind == KIND_P2) p2_unkey(key, &vv, &tt, &r);
    for (size_t k = 0; k < v.size(); ++k)
      if (v[k].group == group && v[k].cfg.kind == kind && v[k].cfg.tt == tt && v[k].cfg.r == r && v[k].cfg.v == vv)
        return (int)k;
    Cls c;
    std::memset(&c.cfg, 0, sizeof(c.cfg));
    c.cfg.kind = kind;
    c.cfg.v = vv;
    c.cfg.tt = tt;
    c.cfg.r = r;
    c.group = group;
    v.push_back(c);
    return (int)v.size() - 1;
  };

  std::map<std::tuple<int, int, int>, long long> hh;  // (M, N, kernel) -> offset
  L.desc.resize(L.B);
  for (int j = 0; j < L.B; ++j) {
    ImageDesc &D = L.desc[j];
    std::memset(&D, 0, sizeof(D));
    D.M = d->rows[j];
    D.N = d->cols[j];
    D.Nh = D.N / 2 + 1;
    D.C = L.C;
    D.kb = (d->ksizes ? d->ksizes[j] : d->ksize) / 2;
    int grb = 0, gw = 0;
    if (!(row_key[j] && col_key[j])) fit_image(D.M, D.N, L.C, L.nt, L.esz, rb_pref, w_pref, &grb, &gw);
    D.Rb = row_key[j] ? p2_rb[grp[j] * kGroupKey + row_key[j]] : grb;
    D.W = col_key[j] ? p2_w[grp[j] * kGroupKey + col_key[j]] : gw;
    D.row_blocks = (D.M + D.Rb - 1) / D.Rb;
    D.col_tiles = (D.Nh + D.W - 1) / D.W;
    Cls &rc = L.row_cls[class_index(L.row_cls, row_key[j] ? KIND_P2 : KIND_GENERIC, row_key[j], grp[j])];
    Cls &cc = L.col_cls[class_index(L.col_cls, col_key[j] ? KIND_P2 : KIND_GENERIC, col_key[j], grp[j])];
    D.row_begin = rc.cfg.grid;
    D.col_begin = cc.cfg.grid;
    rc.cfg.grid += D.row_blocks;
    cc.cfg.grid += L.C * D.col_tiles;
    rc.imgs.push_back(j);
    cc.imgs.push_back(j);
    D.row_pbase = L.total_row_items;
    L.total_row_items += D.row_blocks;
    L.row_grid += D.row_blocks;
    L.col_grid += L.C * D.col_tiles;
    if (row_key[j]) {
      rc.cfg.stage = row_stage;
      rc.cfg.fused = (tune && tune->fused_rows) ? 1 : 0;
      rc.cfg.nt = p2_row_threads(L.C, D.Rb, rc.cfg.tt, rc.cfg.r);
      rc.cfg.smem =
          std::max(rc.cfg.smem, p2_row_smem_half(L.C, D.N, D.Rb, rc.cfg.tt, L.esz, rc.cfg.r, row_stage, 0, rc.cfg.v));
      rc.cfg.smem_fwd = std::max(
          rc.cfg.smem_fwd, p2_row_smem_half(L.C, D.N, D.Rb, rc.cfg.tt, L.esz, rc.cfg.r, row_stage, 1, rc.cfg.v));
    } else {
      rc.cfg.nt = L.nt;
      const size_t ldr = (size_t)((L.C * (D.Rb + 2)) | 1);
      rc.cfg.smem = std::max(rc.cfg.smem, (size_t)D.N * ldr * 2 * L.esz + (size_t)(D.Rb + 1) * D.N * L.esz);
    }
    if (col_key[j]) {
      cc.cfg.nt = p2_col_threads(D.W, cc.cfg.tt, cc.cfg.r);
      cc.cfg.smem = std::max(cc.cfg.smem, p2_col_smem(D.M, D.W, cc.cfg.tt, L.esz, cc.cfg.r, cc.cfg.v));
    } else {
      cc.cfg.nt = L.nt;
      cc.cfg.smem = std::max(cc.cfg.smem, (size_t)D.M * (size_t)((2 * D.W) | 1) * 2 * L.esz);
    }
    rc.cfg.channels = cc.cfg.channels = L.C;
    D.px = L.total_px;
    L.img_px_begin.push_back(L.total_px);
    L.total_px += (long long)L.C * D.M * D.N;
    D.spec = L.total_spec;
    L.total_spec += (long long)L.C * D.M * D.Nh;
    D.mask_plane = ((long long)D.M * D.N + 31) / 32;
    D.mask = L.total_words;
    D.halo = L.total_halo;
    L.total_halo += (long long)L.C * D.N;
    L.img_word_begin.push_back(L.total_words);
    L.total_words += L.C * D.mask_plane;
    for (int c = 0; c < L.C; ++c) {
      L.plane_img.push_back(j);
      L.plane_img.push_back(c);
    }
    const int kidx = L.kernel_per_image ? j : 0;
    auto key = std::make_tuple(D.M, D.N, kidx);
    auto it = hh.find(key);
    if (it == hh.end()) {
      HhatJob job{D.M, D.N, D.Nh, L.K, L.total_hhat, (long long)kidx * L.K * L.K, L.total_g};
      L.g_begin.push_back(L.total_g);
      L.total_g += (long long)L.K * D.Nh;
      L.job_begin.push_back(L.hhat_total_elems);
      L.hhat_total_elems += (long long)D.M * D.Nh;
      L.jobs.push_back(job);
      hh[key] = L.total_hhat;
      D.hhat = L.total_hhat;
      L.total_hhat += (long long)D.M * D.Nh;
    } else {
      D.hhat = it->second;
    }
    for (int len : {D.M, D.N})
      if (!L.tw_off.count(len)) {
        L.tw_off[len] = (int)L.total_tw;
        L.s2_off[len] = (int)L.total_s2;
        L.total_tw += len;
        L.total_s2 += len;
        L.lengths.push_back(len);
      }
    D.tw_row = L.tw_off[D.N];
    D.tw_col = L.tw_off[D.M];
    D.s2_row = L.s2_off[D.N];
    D.s2_col = L.s2_off[D.M];
    // [k1][t] tables of the power-of-two (sub-)lengths and [r][k2] tables of
    // the R * 2^k lengths share one array (tw2_off keyed by length, tw3 by -length).
    D.tw2_row = D.tw2_col = D.tw3_row = D.tw3_col = -1;
    D.tw16_row = D.tw16_col = D.twab_row = D.twab_col = -1;
    for (int pass = 0; pass < 2; ++pass) {
      int tt0, r0;
      if (!reg_fft_params(pass ? D.M : D.N, &tt0, &r0)) continue;
      const int len = 32 * tt0;  // the power-of-two (sub-)length
      // 16 values per thread: [k1][q] table (key len + 2^20), and for L/16 > 16
      // the [a][c] table of the L/16-point stage (key len + 2^21)
      const int k16 = len + (1 << 20), kab = len + (1 << 21), tt16 = len / 16;
      if (!L.tw2_off.count(k16)) {
        L.tw2_off[k16] = (int)L.total_tw2;
        L.total_tw2 += len;
      }
      (pass ? D.tw16_col : D.tw16_row) = L.tw2_off[k16];
      if (tt16 > 16) {
        if (!L.tw2_off.count(kab)) {
          L.tw2_off[kab] = (int)L.total_tw2;
          L.total_tw2 += tt16;
        }
        (pass ? D.twab_col : D.twab_row) = L.tw2_off[kab];
      }
    }
    for (int pass = 0; pass < 2; ++pass) {
      const int len = pass ? D.M : D.N;
      int tt, r;
      if (!reg_fft_params(len, &tt, &r)) continue;
      const int sub = 32 * tt;
      if (!L.tw2_off.count(sub)) {
        L.tw2_off[sub] = (int)L.total_tw2;
        L.total_tw2 += sub;
      }
      if (r > 1 && !L.tw2_off.count(-len)) {
        L.tw2_off[-len] = (int)L.total_tw2;
        L.total_tw2 += len;
      }
      (pass ? D.tw2_col : D.tw2_row) = L.tw2_off[sub];
      if (r > 1) (pass ? D.tw3_col : D.tw3_row) = L.tw2_off[-len];
    }
    factor235(D.N, &D.sched_row);
    factor235(D.M, &D.sched_col);
  }
  L.grp_row.assign(L.ngroups, {});
  L.grp_col.assign(L.ngroups, {});
  for (size_t k = 0; k < L.row_cls.size(); ++k) L.grp_row[L.row_cls[k].group].push_back((int)k);
  for (size_t k = 0; k < L.col_cls.size(); ++k) L.grp_col[L.col_cls[k].group].push_back((int)k);
  for (auto &c : L.row_cls) L.row_smem = std::max(L.row_smem, c.cfg.smem);
  for (auto &c : L.col_cls) L.col_smem = std::max(L.col_smem, c.cfg.smem);
  if (L.row_smem > kMaxSmem || L.col_smem > kMaxSmem) return DECONV_EUNSUPPORTED;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  L.o_yt = take(L.total_px * L.esz);
  L.o_d0 = take(L.total_px * 2 * L.esz);
  L.o_d1 = take(L.total_px * 2 * L.esz);
  L.o_Sa = take(L.total_spec * 4 * L.esz);
  L.o_Sb = take(L.total_spec * 4 * L.esz);
  L.o_hhat = take(L.total_hhat * 2 * L.esz);
  L.o_bits = take(L.total_words * 4);
  L.o_tw = take(L.total_tw * 2 * L.esz);
  L.o_tw2 = take(L.total_tw2 * 2 * L.esz);
  L.o_s2 = take(L.total_s2 * L.esz);
  L.o_desc = take(L.desc.size() * sizeof(ImageDesc));
  L.o_jobs = take(L.jobs.size() * sizeof(HhatJob));
  L.o_jobbeg = take(L.job_begin.size() * sizeof(long long));
  L.o_wordbeg = take(L.img_word_begin.size() * sizeof(long long));
  L.o_pxbeg = take(L.img_px_begin.size() * sizeof(long long));
  L.o_planeimg = take(L.plane_img.size() * sizeof(int));
  L.o_meanpart = take(L.plane_img.size() / 2 * kMeanBlocks * 2 * sizeof(double));
  L.o_means = take(L.plane_img.size() / 2 * sizeof(double));
  L.o_partials = take((size_t)L.total_row_items * 3 * sizeof(double));
  L.o_err = take(sizeof(int));
  L.o_xbuf = take(L.total_px * L.esz);
  // penalty adaptation: v_x (as d), mu / mu_prev / d-rescaling per image, residual partials
  L.o_v = take(L.total_px * 2 * L.esz);
  L.o_mu = take((size_t)3 * L.B * sizeof(double));
  L.o_apart = take((size_t)L.total_row_items * 2 * sizeof(double));
  L.o_halo = take(L.total_halo * L.esz);
  L.o_hg = take((size_t)L.total_g * 16);
  L.o_gbeg = take(L.g_begin.size() * sizeof(long long));
  // fused row pass: per row class a 64-bit ticket counter and a flag per work item
  {
    size_t sync = 0;
    for (auto &c : L.row_cls) {
      c.o_ticket = sync;
      c.o_flags = sync + 8;
      sync = (sync + 8 + 4 * (size_t)c.cfg.grid + 7) / 8 * 8;
    }
    L.sync_bytes = sync;
    L.o_sync = take(sync);
    for (auto &c : L.row_cls) {
      c.o_ticket += L.o_sync;
      c.o_flags += L.o_sync;
    }
  }
  for (auto *v : {&L.row_cls, &L.col_cls})
    for (auto &c : *v) c.o_imgs = take(c.imgs.size() * sizeof(int));
  L.total = o;
  return DECONV_OK;
}

// The tunings deconv_autotune tries: CTAs per register-FFT row class and per
// column pass (a multiple of the 152 SMs, or half of it), and for one channel
// the staged or L1 forward row half.
std::vector<deconv_tune> tune_candidates(int channels) {
  std::vector<deconv_tune> v;
  for (int fv : {16, 32})
    for (int cfv : {16, 32})
      for (int st : channels == 1 ? std::vector<int>{0, 1} : std::vector<int>{0})
        for (int rc : {152, 608})
          for (int cc : {152, 608}) v.push_back(deconv_tune{rc, cc, st, fv, cfv, 0, 0, 0, 0});
  return v;
}

}  // namespace

struct deconv_plan_s {
  Layout L;
  cudaStream_t stream = nullptr;
  char *ws = nullptr;
  double lambda = 0, mu = 1;
  float relax = 2.0f;
  int parity = 0;
  bool have_state = false;
  // Options (deconv_set_options): BGS passes per iteration, Tikhonov warm start, penalty adaptation.
  int passes = 1;
  int tikh_iters = 0;
  double tikh_tau = 1e-3;
  double adapt_t = 0.0;
  bool adapt_ready = false;  // the per-image penalties and v were set by a fresh solve (or a state blob)
  // Creation arguments kept for re-tuning (deconv_retune / deconv_autotune).
  deconv_dims dims{};
  std::vector<int32_t> rows, cols, ksizes;
  size_t ws_bytes = 0;
  deconv_tune tune{0, 0, -1, 0, 0, 0, 0, 0};  // the launch tuning in force (deconv_get_tune)
  long long wait_ns = 2000000000LL;  // bound of every device-side wait (deconv_set_wait_limit)
  cudaGraphExec_t gexec = nullptr;
  // While a graph is captured: the kernel classes of one pass (disjoint sets
  // of images) fan out over side streams, so their launches run concurrently.
  cudaStream_t fan_main = nullptr;
  std::vector<cudaStream_t> fan_side;
  cudaEvent_t fan_fork = nullptr;
  std::vector<cudaEvent_t> fan_join;
  // In-graph pass timing (deconv_set_profiling): events recorded before the
  // first pass and after every pass of the captured loop, in order.
  bool profile = false;
  bool prof_ran = false;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_kind;  // per interval between consecutive events: 0 column pass, 1 row pass

  template <typename P> P *at(size_t off) const { return reinterpret_cast<P *>(ws + off); }
};

namespace {

// Last failing CUDA call of this thread, for deconv_last_error().
thread_local char g_last_error[256] = "";

deconv_status cuda_fail(cudaError_t e, int line) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at plan.cu:%d", cudaGetErrorName(e),
                cudaGetErrorString(e), line);
  return DECONV_ECUDA;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, __LINE__);    \
  } while (0)

template <typename T>
RowArgs<T> row_args(const deconv_plan_s *p, const Cls &c, int mode, const T *d_in, T *d_out, T *x_out,
                    double *partials, double relax) {
  const Layout &L = p->L;
  RowArgs<T> a{};
  a.desc = p->at<ImageDesc>(L.o_desc);
  a.cls_imgs = p->at<int>(c.o_imgs);
  a.nimg = (int)c.imgs.size();
  a.mode = mode;
  a.yt = p->at<T>(L.o_yt);
  a.d_in = d_in;
  a.d_out = d_out;
  a.S_in = p->at<cpair<T>>(L.o_Sb);
  a.S_out = p->at<cpair<T>>(L.o_Sa);
  a.mask = p->at<uint32_t>(L.o_bits);
  a.tw = p->ws + L.o_tw;
  a.tw2 = p->ws + L.o_tw2;
  a.mu = (T)p->mu;
  a.tau = (T)(p->lambda / p->mu);
  a.relax = (T)relax;
  a.lambda = (T)p->lambda;
  a.x_out = x_out;
  a.xbuf = p->at<T>(L.o_xbuf);
  a.partials = partials;
  a.err = p->at<int>(L.o_err);
  a.ticket = p->at<unsigned long long>(c.o_ticket);
  a.flags = p->at<unsigned>(c.o_flags);
  a.halo = p->at<T>(L.o_halo);
  a.items = c.cfg.grid;
  a.wait_ns = p->wait_ns;
  // A state that fits comfortably in the 126 MB L2 stays there from pass to
  // pass; only a larger one gains from the forward half's row prefetch.
  a.prefetch = p->L.total > kL2PrefetchMin ? 1 : 0;
  if (p->adapt_t > 0.0) {
    a.mu_img = p->at<double>(L.o_mu);
    a.mu_prev_img = a.mu_img + L.B;
    a.dscale_img = a.mu_img + 2 * L.B;
    a.vbuf = p->at<T>(L.o_v);
    a.apart = p->at<double>(L.o_apart);
    a.lam64 = p->lambda;
  }
  return a;
}

template <typename T>
ColArgs<T> col_args(const deconv_plan_s *p, const Cls &c, double tikh) {
  const Layout &L = p->L;
  ColArgs<T> a{};
  a.desc = p->at<ImageDesc>(L.o_desc);
  a.cls_imgs = p->at<int>(c.o_imgs);
  a.nimg = (int)c.imgs.size();
  a.S_in = p->at<cpair<T>>(L.o_Sa);
  a.S_out = p->at<cpair<T>>(L.o_Sb);
  a.hhat = p->ws + L.o_hhat;
  a.tw = p->ws + L.o_tw;
  a.tw2 = p->ws + L.o_tw2;
  a.s2 = p->at<T>(L.o_s2);
  a.mu = (T)p->mu;
  a.tikh = (T)tikh;
  a.err = p->at<int>(L.o_err);
  if (p->adapt_t > 0.0) a.mu_img = p->at<double>(L.o_mu);
  return a;
}

template <typename T> T *dbuf(deconv_plan_s *p, int which) {
  return p->at<T>(which ? p->L.o_d1 : p->L.o_d0);
}

// Launches fn(class k, stream) for the classes `idx` of a pass: on s in
// order, or, while a graph is captured on fan_main, the n-th class (n > 0)
// on side stream n-1 (forked from and joined back into s).
template <typename F>
cudaError_t each_class(deconv_plan_s *p, cudaStream_t s, const std::vector<int> &idx, F fn) {
  const size_t n = idx.size();
  const bool fan = n > 1 && s == p->fan_main && p->fan_side.size() + 1 >= n;
  if (fan) {
    cudaError_t e = cudaEventRecord(p->fan_fork, s);
    if (e != cudaSuccess) return e;
  }
  for (size_t k = 0; k < n; ++k) {
    cudaStream_t sk = s;
    if (fan && k > 0) {
      sk = p->fan_side[k - 1];
      cudaError_t e = cudaStreamWaitEvent(sk, p->fan_fork, 0);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = fn((size_t)idx[k], sk);
    if (e != cudaSuccess) return e;
    if (fan && k > 0) {
      e = cudaEventRecord(p->fan_join[k - 1], sk);
      if (e != cudaSuccess) return e;
    }
  }
  if (fan)
    for (size_t k = 1; k < n; ++k) {
      cudaError_t e = cudaStreamWaitEvent(s, p->fan_join[k - 1], 0);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

// Class indices of a pass: those of image group g, or every class (g < 0).
const std::vector<int> &pass_classes(const deconv_plan_s *p, bool row, int g, std::vector<int> &all) {
  const Layout &L = p->L;
  if (g >= 0) return row ? L.grp_row[g] : L.grp_col[g];
  all.resize(row ? L.row_cls.size() : L.col_cls.size());
  for (size_t k = 0; k < all.size(); ++k) all[k] = (int)k;
  return all;
}

// One iteration (column pass then row pass), d ping-pong by plan parity.
// tikh > 0: a Tikhonov warm-start step (denominator |H|^2 + tikh, R ignored).
// g >= 0: the classes of image group g only.
template <typename T>
cudaError_t col_pass(deconv_plan_s *p, cudaStream_t s, double tikh = 0.0, int g = -1) {
  const auto &cl = p->L.col_cls;
  const int ext = (tikh > 0.0 || p->adapt_t > 0.0) ? 1 : 0;  // the column variant with those terms
  std::vector<int> all;
  return each_class(p, s, pass_classes(p, false, g, all), [&](size_t k, cudaStream_t sk) {
    LaunchCfg c = cl[k].cfg;
    c.stage = ext;
    return launch_col<T>(col_args<T>(p, cl[k], tikh), c, sk);
  });
}

// relax < 0: the plan's over-relaxation.  ROW_INNER runs, on the
// register-FFT classes, the inverse half (z-update) and then the forward
// spectrum of y~ alone (row_yspec_p2_kernel).
template <typename T>
cudaError_t row_pass(deconv_plan_s *p, cudaStream_t s, int mode, const T *d_in, T *d_out, T *x_out,
                     double *partials, double relax = -1.0, int g = -1) {
  const auto &cl = p->L.row_cls;
  std::vector<int> all;
  const std::vector<int> &idx = pass_classes(p, true, g, all);
  const double rx = relax < 0.0 ? p->relax : relax;
  const bool adapt = p->adapt_t > 0.0;
  auto cfg_of = [&](size_t k) {
    LaunchCfg c = cl[k].cfg;
    if (adapt) c.stage = 2;  // the forward half with penalty adaptation
    return c;
  };
  if (adapt && mode == ROW_ITER) {
    // Penalty adaptation, Eq. (varying_penalty): z-update and residual norms,
    // the per-image rule, then the forward half with mu^{i+1} and d rescaled.
    const Layout &L = p->L;
    cudaError_t e = each_class(p, s, idx, [&](size_t k, cudaStream_t sk) {
      const LaunchCfg c = cfg_of(k);
      if (c.kind != KIND_P2)
        return launch_row<T>(row_args<T>(p, cl[k], ROW_NORMS, d_in, d_out, x_out, nullptr, rx), c, sk);
      cudaError_t e1 = launch_row_half<T>(row_args<T>(p, cl[k], ROW_ITER, d_in, d_out, x_out, partials, rx), c, 0, sk);
      if (e1 != cudaSuccess) return e1;
      return launch_row_half<T>(row_args<T>(p, cl[k], ROW_NORMS, d_in, d_out, x_out, nullptr, rx), c, 1, sk);
    });
    if (e != cudaSuccess) return e;
    double *mu = p->at<double>(L.o_mu);
    e = launch_mu_update(p->at<ImageDesc>(L.o_desc), L.B, p->at<double>(L.o_apart), mu, mu + L.B, mu + 2 * L.B,
                         p->adapt_t, s);
    if (e != cudaSuccess) return e;
    return each_class(p, s, idx, [&](size_t k, cudaStream_t sk) {
      const LaunchCfg c = cfg_of(k);
      const RowArgs<T> a = row_args<T>(p, cl[k], ROW_ITER, d_in, d_out, x_out, partials, rx);
      if (c.kind != KIND_P2) return launch_row<T>(a, c, sk);
      return launch_row_half<T>(a, c, 1, sk);
    });
  }
  return each_class(p, s, idx, [&](size_t k, cudaStream_t sk) {
    const RowArgs<T> a = row_args<T>(p, cl[k], mode, d_in, d_out, x_out, partials, rx);
    // a plain iteration without statistics: the fused row pass (one kernel)
    if (mode == ROW_ITER && !partials && cl[k].cfg.kind == KIND_P2 && cl[k].cfg.fused)
      return launch_row_half<T>(a, cfg_of(k), 3, sk);
    if (mode == ROW_INNER && cl[k].cfg.kind == KIND_P2) {
      cudaError_t e1 = launch_row_half<T>(a, cfg_of(k), 0, sk);  // z-update
      return e1 != cudaSuccess ? e1 : launch_row_half<T>(a, cfg_of(k), 2, sk);  // y~ spectrum
    }
    return launch_row<T>(a, cfg_of(k), sk);
  });
}

// One iteration of every image (g < 0), or of image group g only (the
// captured loop; the caller flips the d parity once all groups ran it).
// prof: record the profiling events between passes (captured loop).
template <typename T>
deconv_status iterate(deconv_plan_s *p, cudaStream_t s, T *x_out, double *stats, int iters, int it, int g = -1,
                      bool prof = false) {
  const Layout &L = p->L;
  auto mark = [&](int kind) -> cudaError_t {
    if (!prof) return cudaSuccess;
    const size_t n = p->prof_kind.size() + 1;
    if (n >= p->prof_ev.size()) return cudaErrorInvalidValue;
    p->prof_kind.push_back(kind);
    // External: a timed event record node of the graph (a plain record
    // during capture only orders the capture's streams)
    return cudaEventRecordWithFlags(p->prof_ev[n], s, cudaEventRecordExternal);
  };
  // Inner BGS passes: x- and z-steps with v and d (hence the R half of the
  // row-spectral intermediate) held fixed.
  for (int k = 0; k + 1 < p->passes; ++k) {
    CK(col_pass<T>(p, s, 0.0, g));
    CK(mark(0));
    CK(row_pass<T>(p, s, ROW_INNER, nullptr, nullptr, nullptr, nullptr, -1.0, g));
    CK(mark(1));
  }
  CK(col_pass<T>(p, s, 0.0, g));
  CK(mark(0));
  double *partials = stats ? p->at<double>(L.o_partials) : nullptr;
  CK(row_pass<T>(p, s, ROW_ITER, dbuf<T>(p, p->parity), dbuf<T>(p, p->parity ^ 1), x_out, partials, -1.0, g));
  CK(mark(1));
  if (g >= 0) return DECONV_OK;
  p->parity ^= 1;
  if (stats) CK(launch_stats_reduce(p->at<ImageDesc>(L.o_desc), L.B, partials, stats, iters, it, p->at<int>(L.o_err), s));
  return DECONV_OK;
}

template <typename T>
deconv_status init_state(deconv_plan_s *p, const T *y, T *x_out) {
  const Layout &L = p->L;
  cudaStream_t s = p->stream;
  const ImageDesc *desc = p->at<ImageDesc>(L.o_desc);
  CK(launch_means<T>(desc, (int)L.plane_img.size() / 2, p->at<int>(L.o_planeimg), y, p->at<uint32_t>(L.o_bits),
                     p->at<double>(L.o_meanpart), p->at<double>(L.o_means), s));
  CK(launch_init_fill<T>(desc, L.B, L.total_px, p->at<long long>(L.o_pxbeg), y, p->at<uint32_t>(L.o_bits),
                         p->at<double>(L.o_means), L.K, p->at<T>(L.o_yt), s));
  p->parity = 0;
  if (p->adapt_t > 0.0) {
    double *mu = p->at<double>(L.o_mu);
    CK(launch_mu_fill(mu, mu + L.B, mu + 2 * L.B, L.B, p->mu, s));
  }
  const int nt = p->tikh_iters;
  CK(row_pass<T>(p, s, ROW_INIT, nullptr, dbuf<T>(p, 0), nt > 0 ? nullptr : x_out, nullptr));
  // Tikhonov warm start (Eqs. (ini_x)-(ini_z)): x = (H^T H + tau I)^{-1} H^T y~,
  // z = M_z H x (no over-relaxation); the last step leaves x^0 = its x, d^0 = 0.
  for (int k = 0; k < nt; ++k) {
    CK(col_pass<T>(p, s, p->tikh_tau));
    if (k + 1 < nt)
      CK(row_pass<T>(p, s, ROW_INNER, nullptr, nullptr, nullptr, nullptr, 1.0));
    else
      CK(row_pass<T>(p, s, ROW_WARM, nullptr, dbuf<T>(p, 0), x_out, nullptr, 1.0));
  }
  p->have_state = true;
  p->adapt_ready = p->adapt_t > 0.0;
  return DECONV_OK;
}

// The captured loop: kGraphIters iterations of every image.  With several
// image groups (and a fixed penalty: the penalty rule's per-image kernel runs
// over the whole batch) each group runs all its iterations before the next,
// so that its intermediate stays in L2 between passes.
template <typename T>
deconv_status ensure_graph(deconv_plan_s *p) {
  if (p->gexec) return DECONV_OK;
  const Layout &L = p->L;
  const bool grouped = L.ngroups > 1 && !(p->adapt_t > 0.0);
  const bool chains = grouped && L.chains;
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  // Side streams besides cs: one per chain but the first (which runs on
  // cs), or the class fan-out of a pass (its classes but the first).
  size_t lanes = 0;
  if (chains) {
    lanes = (size_t)L.ngroups;
  } else if (grouped) {
    for (int g = 0; g < L.ngroups; ++g)
      lanes = std::max(lanes, std::max(L.grp_row[g].size(), L.grp_col[g].size()));
  } else {
    lanes = std::max(L.row_cls.size(), L.col_cls.size());
  }
  const size_t nside = lanes > 0 ? lanes - 1 : 0;
  deconv_status st = DECONV_OK;
  if (nside > 0) {
    // side streams: the class fan-out of a pass, or one stream per chain
    if (cudaEventCreateWithFlags(&p->fan_fork, cudaEventDisableTiming) != cudaSuccess) st = DECONV_ECUDA;
    for (size_t k = 0; k < nside && st == DECONV_OK; ++k) {
      cudaStream_t sk = nullptr;
      cudaEvent_t ek = nullptr;
      if (cudaStreamCreateWithFlags(&sk, cudaStreamNonBlocking) != cudaSuccess) st = DECONV_ECUDA;
      else p->fan_side.push_back(sk);
      if (cudaEventCreateWithFlags(&ek, cudaEventDisableTiming) != cudaSuccess) st = DECONV_ECUDA;
      else p->fan_join.push_back(ek);
    }
    if (st == DECONV_OK && !chains) p->fan_main = cs;
  }
  // Profiling events: one before the loop and one after every pass.
  for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
  p->prof_ev.clear();
  p->prof_kind.clear();
  p->prof_ran = false;
  if (p->profile && st == DECONV_OK) {
    // chains: the passes of different groups overlap, so only the loop's
    // start and end are marked
    const size_t n = chains ? 2 : (size_t)kGraphIters * (grouped ? L.ngroups : 1) * 2 * p->passes + 1;
    for (size_t k = 0; k < n && st == DECONV_OK; ++k) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) st = DECONV_ECUDA;
      else p->prof_ev.push_back(e);
    }
  }
  const int saved = p->parity;
  p->parity = 0;
  cudaGraph_t g = nullptr;
  if (st == DECONV_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    st = DECONV_ECUDA;
  const bool prof = p->profile && st == DECONV_OK;
  if (prof && cudaEventRecordWithFlags(p->prof_ev[0], cs, cudaEventRecordExternal) != cudaSuccess) st = DECONV_ECUDA;
  if (chains) {
    // each group (one row and one column kernel class) iterates on a stream
    // of its own; the groups share no data, so they join only at the end
    if (st == DECONV_OK && cudaEventRecord(p->fan_fork, cs) != cudaSuccess) st = DECONV_ECUDA;
    if (st == DECONV_OK && p->fan_side.size() + 1 < (size_t)L.ngroups) st = DECONV_ECUDA;  // one stream per chain
    for (int gi = 0; gi < L.ngroups && st == DECONV_OK; ++gi) {
      cudaStream_t sg = gi == 0 ? cs : p->fan_side[gi - 1];
      if (gi > 0 && cudaStreamWaitEvent(sg, p->fan_fork, 0) != cudaSuccess) st = DECONV_ECUDA;
      p->parity = 0;
      for (int k = 0; k < kGraphIters && st == DECONV_OK; ++k) {
        st = iterate<T>(p, sg, nullptr, nullptr, 0, 0, gi, false);
        p->parity ^= 1;
      }
      if (st == DECONV_OK && gi > 0 && cudaEventRecord(p->fan_join[gi - 1], sg) != cudaSuccess) st = DECONV_ECUDA;
    }
    for (int gi = 1; gi < L.ngroups && st == DECONV_OK; ++gi)
      if (cudaStreamWaitEvent(cs, p->fan_join[gi - 1], 0) != cudaSuccess) st = DECONV_ECUDA;
    if (prof && st == DECONV_OK && cudaEventRecordWithFlags(p->prof_ev[1], cs, cudaEventRecordExternal) != cudaSuccess)
      st = DECONV_ECUDA;
  } else if (grouped) {
    for (int gi = 0; gi < L.ngroups && st == DECONV_OK; ++gi) {
      p->parity = 0;
      for (int k = 0; k < kGraphIters && st == DECONV_OK; ++k) {
        st = iterate<T>(p, cs, nullptr, nullptr, 0, 0, gi, prof);
        p->parity ^= 1;
      }
    }
  } else {
    for (int k = 0; k < kGraphIters && st == DECONV_OK; ++k) st = iterate<T>(p, cs, nullptr, nullptr, 0, 0, -1, prof);
  }
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  p->parity = saved;
  p->fan_main = nullptr;
  for (cudaStream_t sk : p->fan_side) cudaStreamDestroy(sk);
  for (cudaEvent_t ek : p->fan_join) cudaEventDestroy(ek);
  if (p->fan_fork) cudaEventDestroy(p->fan_fork);
  p->fan_side.clear();
  p->fan_join.clear();
  p->fan_fork = nullptr;
  if (st == DECONV_OK && e == cudaSuccess && g) {
    if (cudaGraphInstantiate(&p->gexec, g, 0) != cudaSuccess) {
      p->gexec = nullptr;
      st = DECONV_ECUDA;
    }
  } else if (st == DECONV_OK) {
    st = DECONV_ECUDA;
  }
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  return st;
}

template <typename T>
deconv_status run_iters(deconv_plan_s *p, T *x, int iters, double *stats) {
  if (stats) {
    for (int it = 0; it < iters; ++it) {
      deconv_status st = iterate<T>(p, p->stream, it == iters - 1 ? x : nullptr, stats, iters, it);
      if (st != DECONV_OK) return st;
    }
    return DECONV_OK;
  }
  int remaining = iters;
  while (remaining > 1) {
    deconv_status st;
    if (p->parity == 0 && remaining - 1 >= kGraphIters) {
      st = ensure_graph<T>(p);
      if (st != DECONV_OK) return st;
      CK(cudaGraphLaunch(p->gexec, p->stream));
      p->prof_ran = p->profile;
      remaining -= kGraphIters;
    } else {
      st = iterate<T>(p, p->stream, nullptr, nullptr, 0, 0);
      if (st != DECONV_OK) return st;
      --remaining;
    }
  }
  if (remaining == 1) return iterate<T>(p, p->stream, x, nullptr, 0, 0);
  return DECONV_OK;
}

template <typename T>
deconv_status solve_t(deconv_plan_s *p, const void *y, void *x, int iters, int warm, double *stats) {
  if (!warm) {
    deconv_status st = init_state<T>(p, static_cast<const T *>(y), iters == 0 ? static_cast<T *>(x) : nullptr);
    if (st != DECONV_OK) return st;
  }
  return run_iters<T>(p, static_cast<T *>(x), iters, stats);
}

// Shared-memory opt-in of every kernel variant a plan may launch.  Classes
// of different image groups can share one kernel (same transform) with
// different launch shapes: each kernel is opted in once, to the largest
// shared memory any of its classes launches with.
std::vector<LaunchCfg> merged_cfgs(const std::vector<Cls> &cls) {
  std::vector<LaunchCfg> out;
  for (const Cls &c : cls) {
    bool found = false;
    for (LaunchCfg &m : out) {
      const LaunchCfg &a = c.cfg;
      if (m.kind == a.kind && m.channels == a.channels && m.tt == a.tt && m.r == a.r && m.v == a.v &&
          m.stage == a.stage && (a.kind == KIND_P2 || m.nt == a.nt)) {
        m.smem = std::max(m.smem, a.smem);
        m.smem_fwd = std::max(m.smem_fwd, a.smem_fwd);
        found = true;
        break;
      }
    }
    if (!found) out.push_back(c.cfg);
  }
  return out;
}

template <typename T>
cudaError_t prepare_all(const Layout &L) {
  for (const LaunchCfg &c : merged_cfgs(L.row_cls)) {
    cudaError_t e = prepare_row<T>(c);
    if (e == cudaSuccess && c.kind == KIND_P2) {  // the forward half with penalty adaptation
      LaunchCfg d = c;
      d.stage = 2;
      e = prepare_row<T>(d);
    }
    if (e != cudaSuccess) return e;
  }
  for (const LaunchCfg &c : merged_cfgs(L.col_cls)) {
    cudaError_t e = prepare_col<T>(c);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Re-lays out the per-row-block and per-class tables for another tuning.
// The arrays that do not depend on it (state, spectra, H^, tables) keep
// their place and contents; the iteration state does not survive.
template <typename T>
deconv_status retune_t(deconv_plan_s *p, const deconv_tune *t) {
  Layout L2;
  deconv_status st = build_layout(&p->dims, &L2, t);
  if (st != DECONV_OK) return st;
  if (L2.total > p->ws_bytes) return DECONV_ENOMEM;
  const Layout &L = p->L;
  if (L2.o_yt != L.o_yt || L2.o_Sa != L.o_Sa || L2.o_Sb != L.o_Sb || L2.o_hhat != L.o_hhat ||
      L2.o_bits != L.o_bits || L2.o_tw != L.o_tw || L2.o_tw2 != L.o_tw2 || L2.o_s2 != L.o_s2 ||
      L2.o_desc != L.o_desc || L2.total_tw2 != L.total_tw2)
    return DECONV_EUNSUPPORTED;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  p->L = L2;
  cudaStream_t s = p->stream;
  for (const auto *v : {&p->L.row_cls, &p->L.col_cls})
    for (const Cls &c : *v)
      CK(cudaMemcpyAsync(p->ws + c.o_imgs, c.imgs.data(), c.imgs.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->ws + p->L.o_desc, p->L.desc.data(), p->L.desc.size() * sizeof(ImageDesc),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(p->ws + p->L.o_err, 0, sizeof(int), s));
  CK(cudaMemsetAsync(p->ws + p->L.o_sync, 0, p->L.sync_bytes, s));  // new grids: tickets and flags restart
  CK(prepare_all<T>(p->L));
  CK(cudaStreamSynchronize(s));
  p->have_state = false;
  p->adapt_ready = false;
  p->tune = t ? *t : deconv_tune{0, 0, -1, 0, 0, 0, 0, 0, 0};
  return DECONV_OK;
}

template <typename T>
deconv_status setup_t(deconv_plan_s *p, const void *h, const uint8_t *mask) {
  const Layout &L = p->L;
  cudaStream_t s = p->stream;
  // Host tables: twiddles exp(-2 pi i k / L) and 4 sin^2(pi k / L), from
  // double-precision cos/sin, rounded once to T.
  std::vector<T> tw(2 * L.total_tw), s2(L.total_s2);
  for (int len : L.lengths) {
    const int o = L.tw_off.at(len), o2 = L.s2_off.at(len);
    for (int k = 0; k < len; ++k) {
      const double a = 2.0 * M_PI * (double)k / (double)len;
      tw[2 * (o + k)] = (T)std::cos(a);
      tw[2 * (o + k) + 1] = (T)(-std::sin(a));
      const double sn = std::sin(M_PI * (double)k / (double)len);
      s2[o2 + k] = (T)(4.0 * sn * sn);
    }
  }
  // [k1][t] tables of the power-of-two transforms: tw2[k1 TT + t] = exp(-2 pi i t k1 / L);
  // [r][k2] tables of the R * L2 transforms: tw3[r L2 + k2] = exp(-2 pi i r k2 / L).
  std::vector<T> tw2(2 * L.total_tw2);
  for (const auto &kv : L.tw2_off) {
    const int o = kv.second;
    if (kv.first >= (1 << 21)) {  // [a][c] = exp(-2 pi i a c / TT), TT = L / 16 = A B
      const int len = kv.first - (1 << 21), tt = len / 16, A = tt == 64 ? 8 : 4, B = tt / A;
      for (int a = 0; a < A; ++a)
        for (int c = 0; c < B; ++c) {
          const double ang = 2.0 * M_PI * (double)(a * c) / (double)tt;
          tw2[2 * (o + a * B + c)] = (T)std::cos(ang);
          tw2[2 * (o + a * B + c) + 1] = (T)(-std::sin(ang));
        }
    } else if (kv.first >= (1 << 20)) {  // [k1][q] = exp(-2 pi i k1 q / L), k1 < 16, q < L / 16
      const int len = kv.first - (1 << 20), tt = len / 16;
      for (int k1 = 0; k1 < 16; ++k1)
        for (int q = 0; q < tt; ++q) {
          const double ang = 2.0 * M_PI * (double)(k1 * q) / (double)len;
          tw2[2 * (o + k1 * tt + q)] = (T)std::cos(ang);
          tw2[2 * (o + k1 * tt + q) + 1] = (T)(-std::sin(ang));
        }
    } else if (kv.first > 0) {
      const int len = kv.first, tt = len / 32;
      for (int k1 = 0; k1 < 32; ++k1)
        for (int t = 0; t < tt; ++t) {
          const double a = 2.0 * M_PI * (double)(k1 * t) / (double)len;
          tw2[2 * (o + k1 * tt + t)] = (T)std::cos(a);
          tw2[2 * (o + k1 * tt + t) + 1] = (T)(-std::sin(a));
        }
    } else {
      const int len = -kv.first;
      int tt, r;
      reg_fft_params(len, &tt, &r);
      const int L2 = 32 * tt;
      for (int rr = 0; rr < r; ++rr)
        for (int k2 = 0; k2 < L2; ++k2) {
          const double a = 2.0 * M_PI * (double)(rr * k2) / (double)len;
          tw2[2 * (o + rr * L2 + k2)] = (T)std::cos(a);
          tw2[2 * (o + rr * L2 + k2) + 1] = (T)(-std::sin(a));
        }
    }
  }
  CK(cudaMemcpyAsync(p->ws + L.o_tw, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  if (!tw2.empty())
    CK(cudaMemcpyAsync(p->ws + L.o_tw2, tw2.data(), tw2.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  for (const auto *v : {&L.row_cls, &L.col_cls})
    for (const Cls &c : *v)
      CK(cudaMemcpyAsync(p->ws + c.o_imgs, c.imgs.data(), c.imgs.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->ws + L.o_s2, s2.data(), s2.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->ws + L.o_desc, L.desc.data(), L.desc.size() * sizeof(ImageDesc), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->ws + L.o_jobs, L.jobs.data(), L.jobs.size() * sizeof(HhatJob), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->ws + L.o_jobbeg, L.job_begin.data(), L.job_begin.size() * sizeof(long long),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->ws + L.o_wordbeg, L.img_word_begin.data(), L.img_word_begin.size() * sizeof(long long),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->ws + L.o_pxbeg, L.img_px_begin.data(), L.img_px_begin.size() * sizeof(long long),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->ws + L.o_planeimg, L.plane_img.data(), L.plane_img.size() * sizeof(int),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(p->ws + L.o_err, 0, sizeof(int), s));
  CK(cudaMemsetAsync(p->ws + L.o_sync, 0, L.sync_bytes, s));
  CK(cudaMemsetAsync(p->ws + L.o_d0, 0, L.total_px * 2 * L.esz, s));
  CK(cudaMemsetAsync(p->ws + L.o_d1, 0, L.total_px * 2 * L.esz, s));
  CK(cudaMemcpyAsync(p->ws + L.o_gbeg, L.g_begin.data(), L.g_begin.size() * sizeof(long long),
                     cudaMemcpyHostToDevice, s));
  CK(launch_hhat<T>(p->at<HhatJob>(L.o_jobs), (int)L.jobs.size(), L.hhat_total_elems, static_cast<const T *>(h),
                    p->ws + L.o_hhat, p->at<long long>(L.o_jobbeg), p->at<long long>(L.o_gbeg), L.total_g,
                    p->ws + L.o_hg, s));
  CK(launch_pack_mask(p->at<ImageDesc>(L.o_desc), L.B, L.total_words, p->at<long long>(L.o_wordbeg), mask,
                      p->at<uint32_t>(L.o_bits), s));
  CK(prepare_all<T>(L));
  CK(cudaStreamSynchronize(s));
  return DECONV_OK;
}

template <typename T>
deconv_status check_kernels(const void *h, const Layout &L, cudaStream_t s) {
  const int nk = L.kernel_per_image ? L.B : 1;
  std::vector<T> hh((size_t)nk * L.K * L.K);
  CK(cudaMemcpyAsync(hh.data(), h, hh.size() * sizeof(T), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < nk; ++k) {
    double sum = 0.0;
    for (int t = 0; t < L.K * L.K; ++t) {
      const double v = (double)hh[(size_t)k * L.K * L.K + t];
      if (!std::isfinite(v)) return DECONV_EINVAL;
      sum += v;
    }
    if (sum == 0.0) return DECONV_EINVAL;  // zero DC gain: H and D share the constant null vector
  }
  return DECONV_OK;
}

}  // namespace


// ------------------------------------------------------------------ grad ---
namespace {

// Reverse-pass workspace (caller-owned, separate from the plan workspace).
struct GradLayout {
  int k = 1, nck = 0, items = 0;
  int v = 16;                         // values per thread of the adjoint row kernel
  std::vector<int> rb, grid, nt;      // per row class
  std::vector<size_t> smem;
  std::vector<int> adj_begin;         // per image
  size_t o_ckyt, o_ckd, o_ckS, o_segX, o_segD, o_segSpec, o_bbuf, o_ybar, o_ab0, o_ab1, o_Sr0, o_Sr1, o_G, o_tpart,
      o_lpart, o_E, o_res, o_xK, o_adjbeg, total;
};

constexpr int kLossBlocks = 256;

// Shared memory of the reverse row kernel: the staged rows (or the transpose
// tiles of its r groups per row, which reuse them), then one row of N
// complex values per (channel, row).
size_t adj_smem(int C, int N, int rb, int tt, size_t esz, int v, int r) {
  const size_t staged = (size_t)C * (2 * (rb + 2) + 4 * (rb + 1)) * N * esz;
  const int groups = p2_row_threads(C, rb, tt, r) / tt;
  const size_t tiles = (size_t)groups * p2_group_stride_hv(tt, v) * 2 * esz;
  return std::max(staged, tiles) + (size_t)((groups + r - 1) / r) * N * 2 * esz;
}

deconv_status grad_layout(const deconv_plan_s *p, int iters, int k, GradLayout *G) {
  if (p->passes != 1 || p->tikh_iters != 0 || p->adapt_t != 0.0) return DECONV_EUNSUPPORTED;
  const Layout &L = p->L;
  if (iters < 1 || k < 1) return DECONV_EINVAL;
  for (const auto *v : {&L.row_cls, &L.col_cls})
    for (const Cls &c : *v)
      if (c.cfg.kind != KIND_P2) return DECONV_EUNSUPPORTED;  // reverse pass: register-transform lengths only
  G->v = 16;
  G->k = std::min(k, iters);
  G->nck = (iters + G->k - 1) / G->k;
  const int maxthr = L.esz == 4 ? 512 : 256;
  G->adj_begin.assign(L.B, 0);
  G->items = 0;
  for (const Cls &c : L.row_cls) {
    const ImageDesc &D0 = L.desc[c.imgs[0]];
    // the reverse row kernel: v values per thread, r groups of tt threads per row
    const int v = G->v, r = c.cfg.r, tt = D0.N / (v * r);
    int rb = D0.Rb;
    while (rb > 1 && (adj_smem(L.C, D0.N, rb, tt, L.esz, v, r) > kMaxSmem ||
                      p2_row_threads(L.C, rb, tt, r) > maxthr || !p2_groups_ok(p2_row_threads(L.C, rb, tt, r), tt)))
      --rb;
    if (adj_smem(L.C, D0.N, rb, tt, L.esz, v, r) > kMaxSmem || p2_row_threads(L.C, rb, tt, r) > maxthr)
      return DECONV_EUNSUPPORTED;
    int grid = 0;
    for (int j : c.imgs) {
      G->adj_begin[j] = grid;
      grid += (L.desc[j].M + rb - 1) / rb;
    }
    G->rb.push_back(rb);
    G->grid.push_back(grid);
    G->nt.push_back(p2_row_threads(L.C, rb, tt, r));
    G->smem.push_back(adj_smem(L.C, D0.N, rb, tt, L.esz, v, r));
    G->items = std::max(G->items, grid);
  }
  const size_t px = L.total_px * L.esz, spec = L.total_spec * 4 * L.esz;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  G->o_ckyt = take(px * G->nck);
  G->o_ckd = take(2 * px * G->nck);
  G->o_ckS = take(spec * G->nck);
  G->o_segX = take(px * G->k);
  G->o_segD = take(2 * px * (G->k + 1));
  G->o_segSpec = take(spec * G->k);
  G->o_bbuf = take(px);
  G->o_ybar = take(px);
  G->o_ab0 = take(2 * px);
  G->o_ab1 = take(2 * px);
  G->o_Sr0 = take(spec);
  G->o_Sr1 = take(spec);
  G->o_G = take(L.total_spec * 2 * L.esz);
  G->o_tpart = take((size_t)G->items * L.row_cls.size() * sizeof(double));
  G->o_lpart = take(kLossBlocks * sizeof(double));
  int maxKNh = 0;
  for (const ImageDesc &D : L.desc) maxKNh = std::max(maxKNh, L.K * D.Nh);
  G->o_E = take((size_t)maxKNh * 2 * sizeof(double));
  G->o_res = take(4 * sizeof(double));
  G->o_xK = take(px);
  G->o_adjbeg = take(G->adj_begin.size() * sizeof(int));
  G->total = o;
  return DECONV_OK;
}

template <typename T>
// x_true: the loss is the mean squared error of x^{iters} against it; or
// xseed (x_true NULL): dL/dx^{iters} is given (a vector-Jacobian product;
// no loss is computed, loss_h receives 0).
deconv_status grad_t(deconv_plan_s *p, const void *y, const void *x_true, int iters, int k, char *gw,
                     double *loss_h, double *dlambda_h, void *dh, void *x_out, const void *xseed = nullptr) {
  const Layout &L = p->L;
  GradLayout G;
  deconv_status st = grad_layout(p, iters, k, &G);
  if (st != DECONV_OK) return st;
  k = G.k;
  cudaStream_t s = p->stream;
  const size_t px = L.total_px * sizeof(T), spec = L.total_spec * 4 * sizeof(T);
  auto at = [&](size_t off) { return gw + off; };
  CK(cudaMemcpyAsync(at(G.o_adjbeg), G.adj_begin.data(), G.adj_begin.size() * sizeof(int), cudaMemcpyHostToDevice,
                     s));
  {
    // one opt-in per adjoint kernel (row length), to the largest shared
    // memory of the classes (image groups) that launch it
    std::map<int, size_t> adj_smem_of;
    for (size_t c = 0; c < L.row_cls.size(); ++c) {
      size_t &m = adj_smem_of[L.desc[L.row_cls[c].imgs[0]].N];
      m = std::max(m, G.smem[c]);
    }
    for (const auto &kv : adj_smem_of) CK(prepare_adj<T>(kv.first, G.v, L.C, kv.second));
  }

  // Forward run of checkpoint segment c from its checkpoint, storing x_{j+1},
  // d_j and the spectra of every step j of the segment for the reverse pass.
  auto store_segment = [&](int c) -> deconv_status {
    const int s0 = c * k, s1 = std::min(s0 + k, iters);
    CK(cudaMemcpyAsync(p->ws + L.o_yt, at(G.o_ckyt) + c * px, px, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(at(G.o_segD), at(G.o_ckd) + 2 * c * px, 2 * px, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(p->ws + L.o_Sa, at(G.o_ckS) + c * spec, spec, cudaMemcpyDeviceToDevice, s));
    for (int j = s0; j < s1; ++j) {
      const int jj = j - s0;
      for (const Cls &cl : L.col_cls) {
        ColArgs<T> ca = col_args<T>(p, cl, 0.0);
        ca.spec_store = reinterpret_cast<cpair<T> *>(at(G.o_segSpec) + jj * spec);
        CK(launch_col<T>(ca, cl.cfg, s));
      }
      CK(row_pass<T>(p, s, ROW_ITER, reinterpret_cast<const T *>(at(G.o_segD) + 2 * jj * px),
                     reinterpret_cast<T *>(at(G.o_segD) + 2 * (jj + 1) * px),
                     reinterpret_cast<T *>(at(G.o_segX) + jj * px), nullptr));
    }
    return DECONV_OK;
  };

  // 1. Forward with checkpoints of (y~, d, forward spectrum) every k
  // iterations; the last segment runs storing its steps, so the reverse
  // sweep need not recompute it (with k >= iters nothing is recomputed).
  st = init_state<T>(p, static_cast<const T *>(y), nullptr);
  if (st != DECONV_OK) return st;
  for (int c = 0; c < G.nck; ++c) {
    CK(cudaMemcpyAsync(at(G.o_ckyt) + c * px, p->ws + L.o_yt, px, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(at(G.o_ckd) + 2 * c * px, dbuf<T>(p, p->parity), 2 * px, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(at(G.o_ckS) + c * spec, p->ws + L.o_Sa, spec, cudaMemcpyDeviceToDevice, s));
    if (c == G.nck - 1) {
      st = store_segment(c);
      if (st != DECONV_OK) return st;
      break;
    }
    const int n = std::min(k, iters - c * k);
    for (int it = 0; it < n; ++it) {
      st = iterate<T>(p, s, nullptr, nullptr, 0, 0);
      if (st != DECONV_OK) return st;
    }
  }
  // x^{iters} is in the plan's x buffer.
  CK(cudaMemcpyAsync(at(G.o_xK), p->ws + L.o_xbuf, px, cudaMemcpyDeviceToDevice, s));
  if (x_out) CK(cudaMemcpyAsync(x_out, p->ws + L.o_xbuf, px, cudaMemcpyDeviceToDevice, s));
  const long long npx = L.total_px;
  double *res = reinterpret_cast<double *>(at(G.o_res));
  if (x_true) {
    CK(launch_sqerr<T>(reinterpret_cast<const T *>(at(G.o_xK)), static_cast<const T *>(x_true), npx,
                       reinterpret_cast<double *>(at(G.o_lpart)), kLossBlocks, s));
    CK(launch_sum(reinterpret_cast<const double *>(at(G.o_lpart)), kLossBlocks, 1.0 / (double)npx, res, s));
  } else {
    CK(cudaMemsetAsync(res, 0, sizeof(double), s));
  }

  // 2. Reverse sweep, one checkpoint segment at a time.
  CK(cudaMemsetAsync(res + 1, 0, 3 * sizeof(double), s));
  CK(cudaMemsetAsync(at(G.o_G), 0, L.total_spec * 2 * sizeof(T), s));
  CK(cudaMemsetAsync(at(G.o_tpart), 0, (size_t)G.items * L.row_cls.size() * sizeof(double), s));
  int cur = 0;  // ab ping-pong
  const ImageDesc *desc = p->at<ImageDesc>(L.o_desc);
  for (int c = G.nck - 1; c >= 0; --c) {
    const int s0 = c * k, s1 = std::min(s0 + k, iters);
    if (c != G.nck - 1) {  // the last segment's steps are still stored from the forward run
      st = store_segment(c);
      if (st != DECONV_OK) return st;
    }
    // Reverse through the segment.
    for (int j = s1 - 1; j >= s0; --j) {
      const int jj = j - s0;
      const bool start = (j == iters - 1);
      if (!start) {
        // C_{j+1} (first half): inverse row DFT of (bb, T~bb); yb += T~bb.
        for (const Cls &cl : L.row_cls) {
          RowArgs<T> ra = row_args<T>(p, cl, ROW_ADJ, nullptr, nullptr, nullptr, nullptr, p->relax);
          ra.S_in = reinterpret_cast<const cpair<T> *>(at(G.o_Sr1));
          ra.xbuf = reinterpret_cast<T *>(at(G.o_bbuf));
          ra.yt = reinterpret_cast<T *>(at(G.o_ybar));
          CK(launch_row_half<T>(ra, cl.cfg, 0, s));
        }
      }
      // C_{j+1} (second half) and A_j, forward row DFT of tb + i xb.
      for (size_t ci = 0; ci < L.row_cls.size(); ++ci) {
        const Cls &cl = L.row_cls[ci];
        AdjArgs<T> aa{};
        aa.desc = desc;
        aa.cls_imgs = p->at<int>(cl.o_imgs);
        aa.nimg = (int)cl.imgs.size();
        aa.adj_begin = reinterpret_cast<const int *>(at(G.o_adjbeg));
        aa.rb = G.rb[ci];
        aa.mode = start ? ADJ_START : ADJ_STEP;
        aa.bbuf = reinterpret_cast<const T *>(at(G.o_bbuf));
        aa.ab_in = reinterpret_cast<const T *>(at(cur ? G.o_ab1 : G.o_ab0));
        aa.ab_out = reinterpret_cast<T *>(at(cur ? G.o_ab0 : G.o_ab1));
        aa.ybar = reinterpret_cast<T *>(at(G.o_ybar));
        aa.xs = start ? reinterpret_cast<const T *>(at(G.o_xK)) : reinterpret_cast<const T *>(at(G.o_segX) + jj * px);
        aa.ds = reinterpret_cast<const T *>(at(G.o_segD) + 2 * jj * px);
        aa.xtrue = static_cast<const T *>(x_true);
        aa.xseed = static_cast<const T *>(xseed);
        aa.mask = p->at<uint32_t>(L.o_bits);
        aa.tw2 = p->ws + L.o_tw2;
        aa.S_out = reinterpret_cast<cpair<T> *>(at(G.o_Sr0));
        aa.mu = (T)p->mu;
        aa.tau = (T)(p->lambda / p->mu);
        aa.relax = (T)p->relax;
        aa.lscale = (T)(2.0 / (double)npx);
        aa.tpart = reinterpret_cast<double *>(at(G.o_tpart)) + ci * G.items;
        CK(launch_adj<T>(aa, L.desc[cl.imgs[0]].N, G.v, L.C, G.grid[ci], G.nt[ci], G.smem[ci], s));
      }
      cur ^= 1;
      // taub of this step (all classes; unused partial slots stay zero) into res[1], fixed order.
      CK(launch_sum(reinterpret_cast<const double *>(at(G.o_tpart)), G.items * (int)L.row_cls.size(), 1.0, res + 2,
                    s));
      CK(launch_add(res + 1, res + 2, s));
      // B_j: the x-step solve of the adjoint pair and the h-gradient spectrum.
      for (const Cls &cl : L.col_cls) {
        ColArgs<T> ca = col_args<T>(p, cl, 0.0);
        ca.S_in = reinterpret_cast<const cpair<T> *>(at(G.o_Sr0));
        ca.S_out = reinterpret_cast<cpair<T> *>(at(G.o_Sr1));
        ca.spec_fwd = reinterpret_cast<const cpair<T> *>(at(G.o_segSpec) + jj * spec);
        ca.gacc = at(G.o_G);
        CK(launch_col<T>(ca, cl.cfg, s));
      }
    }
  }
  // 3. dL/dh from the spectrum, dL/dlambda = taub / mu.
  const int nk = L.kernel_per_image ? L.B : 1;
  CK(cudaMemsetAsync(dh, 0, (size_t)nk * L.K * L.K * sizeof(T), s));
  for (int j = 0; j < L.B; ++j) {
    T *dhj = static_cast<T *>(dh) + (L.kernel_per_image ? (size_t)j * L.K * L.K : 0);
    CK(launch_taps<T>(desc, j, L.desc[j].M, L.desc[j].N, L.C, L.K, at(G.o_G), reinterpret_cast<double *>(at(G.o_E)), dhj, 1, s));
  }
  double hres[2] = {0, 0};
  CK(cudaMemcpyAsync(hres, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *loss_h = hres[0];
  *dlambda_h = hres[1] / p->mu;
  p->have_state = true;
  return DECONV_OK;
}

}  // namespace

extern "C" deconv_status deconv_grad_workspace_size(deconv_plan p, int32_t iters, int32_t ckpt_every, size_t *bytes) {
  if (!p || !bytes) return DECONV_EINVAL;
  GradLayout G;
  deconv_status st = grad_layout(p, iters, ckpt_every, &G);
  if (st != DECONV_OK) return st;
  *bytes = G.total;
  return DECONV_OK;
}

extern "C" deconv_status deconv_grad(deconv_plan p, const void *y, const void *x_true, int32_t iters,
                                     int32_t ckpt_every, void *grad_ws, size_t grad_ws_bytes, double *loss,
                                     double *dlambda, void *dh, void *x_out) {
  if (!p || !y || !x_true || !grad_ws || !loss || !dlambda || !dh) return DECONV_EINVAL;
  if (reinterpret_cast<uintptr_t>(grad_ws) % kAlign != 0) return DECONV_EINVAL;
  GradLayout G;
  deconv_status st = grad_layout(p, iters, ckpt_every, &G);
  if (st != DECONV_OK) return st;
  if (grad_ws_bytes < G.total) return DECONV_ENOMEM;
  return p->L.dtype == DECONV_F32
             ? grad_t<float>(p, y, x_true, iters, ckpt_every, static_cast<char *>(grad_ws), loss, dlambda, dh, x_out)
             : grad_t<double>(p, y, x_true, iters, ckpt_every, static_cast<char *>(grad_ws), loss, dlambda, dh,
                              x_out);
}

extern "C" deconv_status deconv_vjp(deconv_plan p, const void *y, const void *xbar, int32_t iters,
                                    int32_t ckpt_every, void *grad_ws, size_t grad_ws_bytes, double *dlambda,
                                    void *dh, void *x_out) {
  if (!p || !y || !xbar || !grad_ws || !dlambda || !dh) return DECONV_EINVAL;
  if (reinterpret_cast<uintptr_t>(grad_ws) % kAlign != 0) return DECONV_EINVAL;
  GradLayout G;
  deconv_status st = grad_layout(p, iters, ckpt_every, &G);
  if (st != DECONV_OK) return st;
  if (grad_ws_bytes < G.total) return DECONV_ENOMEM;
  double loss = 0.0;
  return p->L.dtype == DECONV_F32
             ? grad_t<float>(p, y, nullptr, iters, ckpt_every, static_cast<char *>(grad_ws), &loss, dlambda, dh,
                             x_out, xbar)
             : grad_t<double>(p, y, nullptr, iters, ckpt_every, static_cast<char *>(grad_ws), &loss, dlambda, dh,
                              x_out, xbar);
}

extern "C" {

deconv_status deconv_workspace_size(const deconv_dims *dims, size_t *bytes) {
  if (!bytes) return DECONV_EINVAL;
  Layout L;
  deconv_status st = build_layout(dims, &L);
  if (st != DECONV_OK) return st;
  // Room for every tuning the autotuner tries and for the generic passes.
  // They share every array but the per-row-work-item ones (statistics and
  // residual partials, 24 + 16 bytes; fused-pass flags, 4 bytes) and the
  // class lists (at most one row and one column class per image, each list
  // and ticket aligned to 256 bytes): a work item is at least one row, so
  // the default layout plus that much for every row and class bounds them.
  long long rows = 0;
  for (int j = 0; j < dims->batch; ++j) rows += dims->rows[j];
  const size_t extra = (size_t)rows * 44 + (size_t)(2 * dims->batch + 2) * 2 * kAlign + 8 * kAlign;
  *bytes = align_up(L.total + extra);
  return DECONV_OK;
}

deconv_status deconv_plan_create(deconv_plan *out, const deconv_dims *dims, const void *h, const uint8_t *mask,
                                 double lambda, double mu, void *workspace, size_t workspace_bytes, void *stream) {
  if (!out) return DECONV_EINVAL;
  *out = nullptr;
  if (!h || !mask || !workspace) return DECONV_EINVAL;
  if (!(std::isfinite(lambda) && lambda >= 0.0) || !(std::isfinite(mu) && mu > 0.0)) return DECONV_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0) return DECONV_EINVAL;
  deconv_plan_s *p = new (std::nothrow) deconv_plan_s();
  if (!p) return DECONV_ENOMEM;
  deconv_status st = build_layout(dims, &p->L);
  if (st == DECONV_OK && workspace_bytes < p->L.total) st = DECONV_ENOMEM;
  if (st != DECONV_OK) {
    delete p;
    return st;
  }
  p->stream = static_cast<cudaStream_t>(stream);
  p->ws = static_cast<char *>(workspace);
  p->ws_bytes = workspace_bytes;
  p->dims = *dims;
  p->rows.assign(dims->rows, dims->rows + dims->batch);
  p->cols.assign(dims->cols, dims->cols + dims->batch);
  p->dims.rows = p->rows.data();
  p->dims.cols = p->cols.data();
  if (dims->ksizes) {
    p->ksizes.assign(dims->ksizes, dims->ksizes + dims->batch);
    p->dims.ksizes = p->ksizes.data();
  }
  p->lambda = lambda;
  p->mu = mu;
  p->relax = dims->relax;
  st = p->L.dtype == DECONV_F32 ? check_kernels<float>(h, p->L, p->stream) : check_kernels<double>(h, p->L, p->stream);
  if (st == DECONV_OK)
    st = p->L.dtype == DECONV_F32 ? setup_t<float>(p, h, mask) : setup_t<double>(p, h, mask);
  if (st != DECONV_OK) {
    delete p;
    return st;
  }
  *out = p;
  return DECONV_OK;
}

deconv_status deconv_set_options(deconv_plan p, const deconv_options *o) {
  if (!p || !o) return DECONV_EINVAL;
  if (o->bgs_passes < 1 || o->bgs_passes > 64 || o->tikh_iters < 0 || !(o->tikh_tau > 0.0) ||
      !(o->adapt_t == 0.0 || o->adapt_t >= 1.0) || !std::isfinite(o->tikh_tau) || !std::isfinite(o->adapt_t))
    return DECONV_EINVAL;
  if ((o->bgs_passes != p->passes || o->adapt_t != p->adapt_t) && p->gexec) {
    cudaGraphExecDestroy(p->gexec);  // the captured iteration differs
    p->gexec = nullptr;
  }
  if (o->adapt_t != p->adapt_t) p->adapt_ready = false;
  p->passes = o->bgs_passes;
  p->tikh_iters = o->tikh_iters;
  p->tikh_tau = o->tikh_tau;
  p->adapt_t = o->adapt_t;
  return DECONV_OK;
}

deconv_status deconv_retune(deconv_plan p, const deconv_tune *t) {
  if (!p) return DECONV_EINVAL;
  if (t && (t->row_ctas < 0 || t->col_ctas < 0 || t->row_ctas > 65536 || t->col_ctas > 65536 || t->row_stage > 1 ||
            (t->fft_values != 0 && t->fft_values != 16 && t->fft_values != 32) ||
            (t->col_fft_values != 0 && t->col_fft_values != 16 && t->col_fft_values != 32) ||
            t->l2_group_mb < -1 || t->l2_group_mb > 65536 || (t->generic != 0 && t->generic != 1) ||
            (t->fused_rows != 0 && t->fused_rows != 1) || (t->chains != 0 && t->chains != 1)))
    return DECONV_EINVAL;
  return p->L.dtype == DECONV_F32 ? retune_t<float>(p, t) : retune_t<double>(p, t);
}

deconv_status deconv_get_tune(deconv_plan p, deconv_tune *t) {
  if (!p || !t) return DECONV_EINVAL;
  *t = p->tune;
  return DECONV_OK;
}

deconv_status deconv_autotune(deconv_plan p, const void *y, int32_t trial_iters, deconv_tune *best,
                              float *best_ms_per_iter) {
  if (!p || !y || trial_iters < 1 || trial_iters > 100000) return DECONV_EINVAL;
  const bool f32 = p->L.dtype == DECONV_F32;
  // Whole captured loops, so that the image-group schedule is what is timed.
  const int iters = (trial_iters + kGraphIters - 1) / kGraphIters * kGraphIters + 1;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  deconv_tune bt{0, 0, -1, 0, 0, 0, 0};
  float bms = -1.f;
  deconv_status st = DECONV_OK;
  auto trial = [&](const deconv_tune &t) {
    if (deconv_retune(p, &t) != DECONV_OK) return;  // a tuning this plan cannot take
    // fresh solve (builds the CUDA graph), then three timed warm continuations (fastest kept)
    st = f32 ? solve_t<float>(p, y, nullptr, iters, 0, nullptr) : solve_t<double>(p, y, nullptr, iters, 0, nullptr);
    float ms = -1.f;
    for (int rep = 0; rep < 3 && st == DECONV_OK; ++rep) {
      if (cudaEventRecord(e0, p->stream) != cudaSuccess) st = DECONV_ECUDA;
      if (st == DECONV_OK)
        st = f32 ? solve_t<float>(p, nullptr, nullptr, iters, 1, nullptr)
                 : solve_t<double>(p, nullptr, nullptr, iters, 1, nullptr);
      float m = 0.f;
      if (st == DECONV_OK && (cudaEventRecord(e1, p->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                              cudaEventElapsedTime(&m, e0, e1) != cudaSuccess))
        st = DECONV_ECUDA;
      if (st == DECONV_OK && (ms < 0.f || m < ms)) ms = m;
    }
    if (st == DECONV_OK && ms >= 0.f && (bms < 0.f || ms < bms)) {
      bms = ms;
      bt = t;
    }
  };
  // Launch shapes first.  The staged forward half (188 KB of shared memory
  // per CTA at 1024) keeps the kernel classes of a batch from running side
  // by side; it is tried for plans of one row class only.
  const bool one_class = p->L.row_cls.size() == 1;
  std::vector<deconv_tune> cands{deconv_tune{0, 0, -1, 0, 0, 0, 0, 0, 0}};  // the defaults
  for (const deconv_tune &t : tune_candidates(p->L.C))
    if (t.row_stage != 1 || one_class) cands.push_back(t);
  for (size_t k = 0; k < cands.size() && st == DECONV_OK; ++k) trial(cands[k]);
  // Then the shared-memory (Stockham) passes, for a small problem: there the
  // register transforms give each row or column only L/16 or L/32 threads
  // (4 for a 64-point FP64 row) and run long dependent chains per thread.
  long long px = 0;
  for (size_t b = 0; b < p->rows.size(); ++b) px += (long long)p->rows[b] * p->cols[b] * p->L.C;
  if (st == DECONV_OK && bms >= 0.f && px <= (1LL << 20)) {
    deconv_tune t = bt;
    t.generic = 1;
    trial(t);
  }
  // Then the image-group budget of the captured loop, for a batch.
  if (st == DECONV_OK && bms >= 0.f && p->L.B > 1 && !(p->adapt_t > 0.0)) {
    const deconv_tune shape = bt;
    for (int mb : {24, 48, 80}) {
      if (st != DECONV_OK) break;
      deconv_tune t = shape;
      t.l2_group_mb = mb;
      trial(t);
    }
  }
  // Then independent chains per kernel class, for a batch.
  if (st == DECONV_OK && bms >= 0.f && p->L.B > 1 && !(p->adapt_t > 0.0)) {
    deconv_tune t = bt;
    t.l2_group_mb = 0;
    t.chains = 1;
    trial(t);
  }
  // Then the fused row pass instead of the two row kernels.
  if (st == DECONV_OK && bms >= 0.f) {
    deconv_tune t = bt;
    t.fused_rows = 1;
    trial(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DECONV_OK) return st;
  if (bms < 0.f) return DECONV_EUNSUPPORTED;
  st = deconv_retune(p, &bt);
  if (st != DECONV_OK) return st;
  if (best) *best = bt;
  if (best_ms_per_iter) *best_ms_per_iter = bms / (float)iters;
  return DECONV_OK;
}

deconv_status deconv_fast_shape(int32_t M, int32_t N, int32_t channels, int32_t ksize, int32_t dtype,
                                int32_t *M_out, int32_t *N_out) {
  if (!M_out || !N_out || M < 1 || N < 1 || (channels != 1 && channels != 3) || ksize < 1 || !(ksize & 1) ||
      (dtype != DECONV_F32 && dtype != DECONV_F64) || M < ksize || N < ksize)
    return DECONV_EINVAL;
  // The first few 2-3-5-smooth lengths at or above each side.
  auto smooth_from = [](int L, int count) {
    std::vector<int> v;
    FftSched sc;
    for (long long c = L; (int)v.size() < count && c <= (1 << 20); ++c)
      if (factor235((int)c, &sc)) v.push_back((int)c);
    return v;
  };
  const std::vector<int> ms = smooth_from(M, 12), ns = smooth_from(N, 12);
  long long best = -1;
  for (int m2 : ms)
    for (int n2 : ns) {
      const long long area = (long long)m2 * n2;
      if (best >= 0 && area >= best) continue;
      int32_t r = m2, c = n2;
      deconv_dims d{};
      d.batch = 1;
      d.channels = channels;
      d.rows = &r;
      d.cols = &c;
      d.ksize = ksize;
      d.dtype = dtype;
      d.relax = 2.0f;
      Layout L;
      if (build_layout(&d, &L) != DECONV_OK) continue;
      best = area;
      *M_out = m2;
      *N_out = n2;
    }
  return best >= 0 ? DECONV_OK : DECONV_EUNSUPPORTED;
}

deconv_status deconv_get_mu(deconv_plan p, double *mu_host) {
  if (!p || !mu_host) return DECONV_EINVAL;
  if (!(p->adapt_t > 0.0 && p->adapt_ready)) {
    for (int j = 0; j < p->L.B; ++j) mu_host[j] = p->mu;
    return DECONV_OK;
  }
  CK(cudaMemcpyAsync(mu_host, p->ws + p->L.o_mu, sizeof(double) * p->L.B, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return DECONV_OK;
}

deconv_status deconv_solve(deconv_plan p, const void *y, void *x, int32_t iters, int32_t warm, double *stats) {
  if (!p || iters < 0 || (warm != 0 && warm != 1)) return DECONV_EINVAL;
  if (!warm && !y) return DECONV_EINVAL;
  if (warm && !p->have_state) return DECONV_EINVAL;
  if (warm && p->adapt_t > 0.0 && !p->adapt_ready) return DECONV_EINVAL;  // no per-image penalties yet
  if (iters > 0 && !x) return DECONV_EINVAL;
  if (stats && iters == 0) stats = nullptr;
  return p->L.dtype == DECONV_F32 ? solve_t<float>(p, y, x, iters, warm, stats)
                                  : solve_t<double>(p, y, x, iters, warm, stats);
}

deconv_status deconv_solve_host(deconv_plan p, const void *y_host, void *x_host, int32_t iters) {
  if (!p || !y_host || !x_host || iters < 0) return DECONV_EINVAL;
  const Layout &L = p->L;
  const size_t bytes = L.total_px * L.esz;
  CK(cudaMemcpyAsync(p->ws + L.o_yt, y_host, bytes, cudaMemcpyHostToDevice, p->stream));
  // y is staged in the y~ buffer itself: the initial fill only rewrites
  // unobserved entries and reads observed ones.
  deconv_status st = p->L.dtype == DECONV_F32
                         ? solve_t<float>(p, p->ws + L.o_yt, p->ws + L.o_xbuf, iters, 0, nullptr)
                         : solve_t<double>(p, p->ws + L.o_yt, p->ws + L.o_xbuf, iters, 0, nullptr);
  if (st != DECONV_OK) return st;
  CK(cudaMemcpyAsync(x_host, p->ws + L.o_xbuf, bytes, cudaMemcpyDeviceToHost, p->stream));
  return deconv_sync(p);
}

deconv_status deconv_set_wait_limit(deconv_plan p, int64_t ns) {
  if (!p || ns < 0) return DECONV_EINVAL;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);  // the bound is a kernel argument of the captured launches
    p->gexec = nullptr;
  }
  p->wait_ns = (long long)ns;
  return DECONV_OK;
}

deconv_status deconv_set_profiling(deconv_plan p, int32_t on) {
  if (!p || (on != 0 && on != 1)) return DECONV_EINVAL;
  if ((on != 0) != p->profile && p->gexec) {
    cudaGraphExecDestroy(p->gexec);  // re-captured with (or without) the events
    p->gexec = nullptr;
  }
  p->profile = on != 0;
  p->prof_ran = false;
  return DECONV_OK;
}

deconv_status deconv_graph_pass_times(deconv_plan p, float *ms_host) {
  if (!p || !ms_host || !p->profile || !p->prof_ran || p->prof_ev.size() < 2) return DECONV_EINVAL;
  if (p->prof_kind.empty()) {  // chains: only the whole loop is timed
    float all = 0.f;
    CK(cudaStreamSynchronize(p->stream));
    CK(cudaEventElapsedTime(&all, p->prof_ev.front(), p->prof_ev.back()));
    ms_host[0] = ms_host[1] = -1.f;
    ms_host[2] = all / (float)kGraphIters;
    return DECONV_OK;
  }
  if (p->prof_ev.size() != p->prof_kind.size() + 1) return DECONV_EINVAL;
  CK(cudaStreamSynchronize(p->stream));
  double t[2] = {0.0, 0.0};
  for (size_t k = 0; k < p->prof_kind.size(); ++k) {
    float m = 0.f;
    CK(cudaEventElapsedTime(&m, p->prof_ev[k], p->prof_ev[k + 1]));
    t[p->prof_kind[k]] += m;
  }
  float all = 0.f;
  CK(cudaEventElapsedTime(&all, p->prof_ev.front(), p->prof_ev.back()));
  ms_host[0] = (float)(t[0] / kGraphIters);
  ms_host[1] = (float)(t[1] / kGraphIters);
  ms_host[2] = all / (float)kGraphIters;
  return DECONV_OK;
}

deconv_status deconv_profile_passes(deconv_plan p, int32_t iters, float *ms_host) {
  if (!p || iters < 1 || !ms_host || !p->have_state) return DECONV_EINVAL;
  std::vector<cudaEvent_t> ev(4 * (size_t)iters, nullptr);
  deconv_status st = DECONV_OK;
  for (auto &e : ev)
    if (st == DECONV_OK && cudaEventCreate(&e) != cudaSuccess) st = DECONV_ECUDA;
  for (int it = 0; it < iters && st == DECONV_OK; ++it) {
    cudaError_t e = cudaEventRecord(ev[4 * it], p->stream);
    const bool f32 = p->L.dtype == DECONV_F32;
    if (e == cudaSuccess) e = f32 ? col_pass<float>(p, p->stream) : col_pass<double>(p, p->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4 * it + 1], p->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4 * it + 2], p->stream);
    if (e == cudaSuccess)
      e = f32 ? row_pass<float>(p, p->stream, ROW_ITER, dbuf<float>(p, p->parity), dbuf<float>(p, p->parity ^ 1),
                                nullptr, nullptr)
              : row_pass<double>(p, p->stream, ROW_ITER, dbuf<double>(p, p->parity),
                                 dbuf<double>(p, p->parity ^ 1), nullptr, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4 * it + 3], p->stream);
    if (e != cudaSuccess) st = DECONV_ECUDA;
    p->parity ^= 1;
  }
  if (st == DECONV_OK && cudaStreamSynchronize(p->stream) != cudaSuccess) st = DECONV_ECUDA;
  double col = 0.0, row = 0.0;
  for (int it = 0; it < iters && st == DECONV_OK; ++it) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, ev[4 * it], ev[4 * it + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&b, ev[4 * it + 2], ev[4 * it + 3]) != cudaSuccess)
      st = DECONV_ECUDA;
    col += a;
    row += b;
  }
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  if (st != DECONV_OK) return st;
  ms_host[0] = (float)(col / iters);
  ms_host[1] = (float)(row / iters);
  return DECONV_OK;
}

deconv_status deconv_sync(deconv_plan p) {
  if (!p) return DECONV_EINVAL;
  int err = 0;
  CK(cudaMemcpyAsync(&err, p->ws + p->L.o_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (err) {
    CK(cudaMemsetAsync(p->ws + p->L.o_err, 0, sizeof(int), p->stream));
    CK(cudaStreamSynchronize(p->stream));
    return (err & 2) ? DECONV_ETIMEOUT : DECONV_ENONFINITE;
  }
  return DECONV_OK;
}

deconv_status deconv_plan_destroy(deconv_plan p) {
  if (!p) return DECONV_EINVAL;
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
  delete p;
  return DECONV_OK;
}

// State blob: y~ | d | forward row spectra | per-image mu, mu_prev, d scale |
// v | flag (int32, padded to 16 bytes).  The penalties and v are the state of
// penalty adaptation; the flag is 1 when they were live in the saving plan.
struct StateParts {
  size_t yt, d, sa, mu, v, total;
};

static StateParts state_parts(const deconv_plan_s *p) {
  StateParts s;
  s.yt = p->L.total_px * p->L.esz;
  s.d = 2 * s.yt;
  s.sa = p->L.total_spec * 4 * p->L.esz;
  s.mu = 3 * (size_t)p->L.B * sizeof(double);
  s.v = 2 * s.yt;
  s.total = s.yt + s.d + s.sa + s.mu + s.v + 16;
  return s;
}

deconv_status deconv_state_bytes(deconv_plan p, size_t *bytes) {
  if (!p || !bytes) return DECONV_EINVAL;
  *bytes = state_parts(p).total;
  return DECONV_OK;
}

deconv_status deconv_state_get(deconv_plan p, void *blob) {
  if (!p || !blob || (reinterpret_cast<uintptr_t>(blob) & 15)) return DECONV_EINVAL;
  if (!p->have_state) return DECONV_EINVAL;
  const StateParts s = state_parts(p);
  const Layout &L = p->L;
  char *o = static_cast<char *>(blob);
  const int32_t flag[4] = {p->adapt_t > 0.0 && p->adapt_ready ? 1 : 0, 0, 0, 0};
  CK(cudaMemcpyAsync(o, p->ws + L.o_yt, s.yt, cudaMemcpyDeviceToDevice, p->stream));
  o += s.yt;
  CK(cudaMemcpyAsync(o, p->ws + (p->parity ? L.o_d1 : L.o_d0), s.d, cudaMemcpyDeviceToDevice, p->stream));
  o += s.d;
  CK(cudaMemcpyAsync(o, p->ws + L.o_Sa, s.sa, cudaMemcpyDeviceToDevice, p->stream));
  o += s.sa;
  CK(cudaMemcpyAsync(o, p->ws + L.o_mu, s.mu, cudaMemcpyDeviceToDevice, p->stream));
  o += s.mu;
  CK(cudaMemcpyAsync(o, p->ws + L.o_v, s.v, cudaMemcpyDeviceToDevice, p->stream));
  o += s.v;
  // From pageable memory: the call returns once the 16 bytes are staged.
  CK(cudaMemcpyAsync(o, flag, sizeof(flag), cudaMemcpyHostToDevice, p->stream));
  return DECONV_OK;
}

deconv_status deconv_state_set(deconv_plan p, const void *blob) {
  if (!p || !blob || (reinterpret_cast<uintptr_t>(blob) & 15)) return DECONV_EINVAL;
  const StateParts s = state_parts(p);
  const Layout &L = p->L;
  const char *o = static_cast<const char *>(blob);
  int32_t flag[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(p->ws + L.o_yt, o, s.yt, cudaMemcpyDeviceToDevice, p->stream));
  o += s.yt;
  CK(cudaMemcpyAsync(p->ws + L.o_d0, o, s.d, cudaMemcpyDeviceToDevice, p->stream));
  o += s.d;
  CK(cudaMemcpyAsync(p->ws + L.o_Sa, o, s.sa, cudaMemcpyDeviceToDevice, p->stream));
  o += s.sa;
  CK(cudaMemcpyAsync(p->ws + L.o_mu, o, s.mu, cudaMemcpyDeviceToDevice, p->stream));
  o += s.mu;
  CK(cudaMemcpyAsync(p->ws + L.o_v, o, s.v, cudaMemcpyDeviceToDevice, p->stream));
  o += s.v;
  CK(cudaMemcpyAsync(flag, o, sizeof(flag), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  p->parity = 0;
  p->have_state = true;
  // A blob without a live adaptive state leaves a warm solve under adaptation refused.
  p->adapt_ready = p->adapt_t > 0.0 && flag[0] == 1;
  return DECONV_OK;
}

deconv_status deconv_kernel_launches(deconv_plan p, int32_t iters, int32_t mode, int32_t ckpt_every,
                                     int64_t *count) {
  if (!p || !count || iters < 0 || (mode != 0 && mode != 1)) return DECONV_EINVAL;
  const Layout &L = p->L;
  long long row = 0, col = (long long)L.col_cls.size();
  long long row_init = 0;  // the initial row pass always runs the two halves
  for (const Cls &c : L.row_cls) {
    row_init += c.cfg.kind == KIND_P2 ? 2 : 1;
    row += c.cfg.kind != KIND_P2 ? 1 : ((c.cfg.fused && p->adapt_t <= 0.0) ? 1 : 2);
  }
  long long inner = 0;  // an inner BGS pass: the inverse half and the y~ spectrum on register-FFT classes
  for (const Cls &c : L.row_cls) inner += c.cfg.kind == KIND_P2 ? 2 : 1;
  // observed means (2 kernels), initial fill, initial row pass, warm-start steps
  const long long init = 3 + row_init + (p->tikh_iters > 0 ? (long long)p->tikh_iters * col +
                                                                 (long long)(p->tikh_iters - 1) * inner + row_init
                                                           : 0);
  long long adapt = 0;  // penalty adaptation: a residual-norm launch per class and the per-image rule
  if (p->adapt_t > 0.0) adapt = (long long)L.row_cls.size() + 1;
  const long long per_iter = col + row + adapt + (long long)(p->passes - 1) * (col + inner);
  if (mode == 0) {
    *count = init + (long long)iters * per_iter;
    return DECONV_OK;
  }
  if (iters < 1 || ckpt_every < 1) return DECONV_EINVAL;
  const long long nrc = (long long)L.row_cls.size();
  // forward + loss (2) + recompute (every segment but the last, stored by the
  // forward run) + reverse per step: inverse halves (not on the first),
  // adjoint stencils, 2 reductions, column passes; taps (2 per image).
  const int k = std::min(ckpt_every, iters), nck = (iters + k - 1) / k;
  const long long recompute = (long long)(nck - 1) * k;
  *count = init + (long long)iters * per_iter + 2 + recompute * per_iter +
           (long long)(iters - 1) * nrc + (long long)iters * (nrc + 2 + col) + 2LL * L.B;
  return DECONV_OK;
}

const char *deconv_last_error(void) { return g_last_error; }

const char *deconv_status_string(deconv_status s) {
  switch (s) {
    case DECONV_OK: return "ok";
    case DECONV_EINVAL: return "invalid argument";
    case DECONV_EUNSUPPORTED: return "unsupported size";
    case DECONV_ENOMEM: return "workspace too small";
    case DECONV_ECUDA: return "CUDA runtime error";
    case DECONV_ETIMEOUT: return "device wait timed out";
    case DECONV_ENONFINITE: return "non-finite value in the iterate";
  }
  return "unknown status";
}

}  // extern "C"
