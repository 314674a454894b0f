// Internal types shared by the device kernels and the host plan code.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fft.cuh"

namespace dcv {

// Per-image geometry and workspace offsets.  Offsets are in elements of the
// array they index (see Plan in plan.cu for the arrays).
struct ImageDesc {
  int M, N, Nh, C;       // extended rows, cols, N/2+1, channels
  int kb;                // half support b of the image's kernel (boundary band of the initial fill)
  int Rb;                // rows owned by one row-pass CTA
  int W;                 // spectral columns (k2) per column-pass CTA
  int row_blocks;        // ceil(M / Rb)
  int col_tiles;         // ceil(Nh / W) (per channel)
  int row_begin;         // first row-pass work item of this image within its kernel class
  int col_begin;         // first column-pass work item (C * col_tiles items) within its class
  int row_pbase;         // first row-pass work item over the whole plan (statistics partials)
  long long px;          // first pixel (real element) of the image, batch layout
  long long spec;        // first cpair of the image in the spectral buffers
  long long hhat;        // first complex of the image's H^ half-spectrum
  long long mask;        // first 32-bit word of the image's packed mask
  long long mask_plane;  // words per channel plane
  long long halo;        // first element of the image's halo row (C x N: x of row M - 1, fused row pass)
  int tw_row, tw_col;    // twiddle-table offsets for lengths N and M
  int s2_row, s2_col;    // 4 sin^2(pi k / L) table offsets for N and M
  int tw2_row, tw2_col;  // [k1][t] twiddle-table offsets of the power-of-two (sub-)length, -1 if none
  int tw3_row, tw3_col;  // [r][k2] twiddles exp(-2 pi i r k2 / L) of a length R * 2^k, -1 if none
  int tw16_row, tw16_col;  // 16 values per thread: [k1][q] twiddles exp(-2 pi i k1 q / L), -1 if none
  int twab_row, twab_col;  // 16 values per thread, L >= 512: [a][c] twiddles exp(-2 pi i a c / (L/16))
  FftSched sched_row, sched_col;
};

// Pair of complex values stored per (row, k2) in the spectral buffers:
// forward: (Y_row, R_row) = row spectra of y~ and r; inverse: (X_row, HX_row).
template <typename T> struct alignas(4 * sizeof(T)) cpair { T ar, ai, br, bi; };

// ROW_ITER: one iteration's row pass.  ROW_INIT: the initial state from y~0.
// ROW_ADJ: reverse pass.  ROW_INNER: an inner block-Gauss-Seidel pass (and a
// Tikhonov warm-start step): z-update, then the row spectrum of y~ alone into
// the Y half of the row-spectral intermediate (the R half is kept).
// ROW_WARM: the last warm-start step: z-update, then the initial state with
// x^0 = the x just computed (d^0 = 0, v^0 = D x^0).
// ROW_NORMS (penalty adaptation): the prox of the forward half only, for the
// per-image residual norms ||d^{i+1} - d^i||^2 and ||v^{i+1} - v^i||^2 (no
// z-update, no d or spectrum written; v^{i+1} replaces v^i in vbuf).
enum RowMode { ROW_ITER = 0, ROW_INIT = 1, ROW_ADJ = 2, ROW_INNER = 3, ROW_WARM = 4, ROW_NORMS = 5 };

template <typename T> struct RowArgs {
  const ImageDesc *desc;
  const int *cls_imgs;    // images of the launched kernel class, by increasing row_begin
  int nimg;               // entries of cls_imgs
  int mode;           // RowMode
  T *yt;              // y~ (observed: y, unobserved: z), batch layout
  const T *d_in;      // d_x^i as (d_h, d_v) pairs per pixel; NULL = zero
  T *d_out;           // d_x^{i+1}
  const cpair<T> *S_in;   // (X_row, HX_row) from the column pass (ROW_ITER)
  cpair<T> *S_out;        // (Y_row, R_row) for the next column pass
  const uint32_t *mask;   // packed observed bits
  const void *tw;         // twiddle tables (cx<T>)
  const void *tw2;        // [k1][t] twiddle tables of the power-of-two transforms (cx<T>)
  T mu, tau, relax, lambda;
  T *x_out;               // nullable: x^{i+1} for owned rows
  T *xbuf;                // plan's x buffer (power-of-two row passes: written by the inverse half)
  // Penalty adaptation (all NULL when mu is fixed): per image mu^{i+1} (mu^i
  // during ROW_NORMS), mu^i, and the rescaling s = mu^i / mu^{i+1} of d^{i+1};
  // v_x per pixel as d; residual-norm partials (2 doubles per row block).
  const double *mu_img, *mu_prev_img, *dscale_img;
  T *vbuf;
  double *apart;
  double lam64;           // lambda in double (tau = lambda / mu per image)
  double *partials;       // nullable: per work item [3] = sum dd^2, dz^2, J
  int *err;
  // Fused row pass (row_fused_p2_kernel): the class's ticket counter and
  // one flag per work item, the halo rows, the items of one launch and the
  // bound of every wait in nanoseconds.
  unsigned long long *ticket;
  unsigned *flags;
  T *halo;
  int items;
  long long wait_ns;
  int prefetch;  // forward half: L2 prefetch of the block's input rows (the state does not fit L2)
};

template <typename T> struct ColArgs {
  const ImageDesc *desc;
  const int *cls_imgs;
  int nimg;
  const cpair<T> *S_in;
  cpair<T> *S_out;
  const void *hhat;   // cx<T>
  const void *tw;     // cx<T>
  const void *tw2;    // cx<T>, [k1][t] layout
  const T *s2;        // 4 sin^2 tables
  T mu;
  T tikh;             // > 0: Tikhonov warm-start step, X = conj(H) Y / (|H|^2 + tikh) (R ignored)
  const double *mu_img;  // nullable: per-image mu (penalty adaptation)
  int *err;
  // Reverse pass only (power-of-two column pass):
  cpair<T> *spec_store;       // nullable: store (Y^, R^) after the forward column DFTs
  const cpair<T> *spec_fwd;   // nullable: forward (Y^, R^) of the same step, with gacc
  void *gacc;                 // cx<T> per (channel, k1, k2): accumulated h-gradient spectrum
};

// One launch of a pass over the images of one kernel class.
enum KernelKind { KIND_GENERIC = 0, KIND_P2 = 1 };
struct LaunchCfg {
  int kind;      // KernelKind
  int tt;        // KIND_P2: threads per sub-transform (sub-length / v)
  int r;         // KIND_P2: length = r * v * tt, r in {1, 3, 5}
  int v;         // KIND_P2: complex values per thread, 32 (fft_p2 / fft_mixed) or 16 (fft_v16, r = 1)
  int stage;     // KIND_P2 rows, forward half: 0 reads through L1, 1 stages its rows (one
                 // channel), 2 reads through L1 with penalty adaptation.  KIND_P2
                 // columns: 1 = the variant with the Tikhonov step / per-image penalty
  int nt;        // threads per CTA
  int channels;  // 1 or 3
  int grid;      // CTAs
  size_t smem;   // dynamic shared memory per CTA
  size_t smem_fwd;  // KIND_P2 rows: the forward half's (smem is the inverse half's)
  int fused;        // KIND_P2 rows: plain iterations run the fused row pass (one kernel)
};

// Kernel launchers (kernels_*.cu).
template <typename T>
cudaError_t launch_row(const RowArgs<T> &a, const LaunchCfg &c, cudaStream_t s);
template <typename T>
cudaError_t launch_col(const ColArgs<T> &a, const LaunchCfg &c, cudaStream_t s);
template <typename T>
cudaError_t prepare_row(const LaunchCfg &c);
template <typename T>
cudaError_t prepare_col(const LaunchCfg &c);

// Reverse pass (adjoint.cu, adjoint.cuh).
enum AdjMode { ADJ_START = 0, ADJ_STEP = 1 };

template <typename T> struct AdjArgs {
  const ImageDesc *desc;
  const int *cls_imgs;
  int nimg;
  const int *adj_begin;  // per image: first work item of this launch
  int rb;                // rows per CTA
  int mode;              // AdjMode
  const T *bbuf;         // bb of step j+1 (ADJ_STEP)
  const T *ab_in;        // ab of step j+1, (h, v) pairs (ADJ_STEP)
  T *ab_out;             // ab of step j
  T *ybar;               // in: yb of step j+1 (after C_{j+1}'s T~bb); out: yb'_j
  const T *xs;           // x_{j+1}
  const T *ds;           // d_j pairs
  const T *xtrue;        // ADJ_START: ground truth for dL/dx (loss = mean squared error)
  const T *xseed;        // ADJ_START, nullable: dL/dx^{iters} given by the caller (replaces xtrue)
  const uint32_t *mask;
  const void *tw2;
  cpair<T> *S_out;       // row spectra of tb + i xb
  T mu, tau, relax, lscale;  // lscale = 2 / (number of pixels in the loss)
  double *tpart;         // per work item: partial taub
};


// The reverse-pass row kernel of a row length 3 * 2^k or 5 * 2^k with v = 16
// values per thread (adjoint_r35.cu; launch and shared-memory opt-in must use
// the pointer it returns); NULL for any other length.
template <typename T>
const void *adj_ptr_r35(int N, int v, int C);
// Reverse-pass row kernel for rows of length N with v complex values per thread (16 or 32).
template <typename T>
cudaError_t launch_adj(const AdjArgs<T> &a, int N, int v, int C, int grid, int nt, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t prepare_adj(int N, int v, int C, size_t smem);
template <typename T>
cudaError_t launch_row_half(const RowArgs<T> &a, const LaunchCfg &c, int half, cudaStream_t s);
template <typename T>
cudaError_t launch_sqerr(const T *x, const T *xt, long long n, double *part, int blocks, cudaStream_t s);
cudaError_t launch_sum(const double *v, int n, double scale, double *out, cudaStream_t s);
cudaError_t launch_add(double *acc, const double *v, cudaStream_t s);
template <typename T>
cudaError_t launch_taps(const ImageDesc *desc, int img, int M, int N, int C, int K, const void *G, double *E,
                        void *dh, int accumulate, cudaStream_t s);

// Setup kernels (setup.cu).
struct HhatJob {          // one half-spectrum to compute
  int M, N, Nh, K;
  long long out;          // complex offset in hhat
  long long h;            // element offset of the kernel
  long long g;            // offset of the job's K x Nh row sums in the double2 scratch
};
// Row sums into G (total_g double2 over all jobs, g_begin per job), then the
// half-spectra (total elements, job_begin per job).
template <typename T>
cudaError_t launch_hhat(const HhatJob *jobs_dev, int njobs, long long total, const T *h, void *hhat,
                        const long long *job_begin_dev, const long long *g_begin_dev, long long total_g, void *G,
                        cudaStream_t s);
cudaError_t launch_pack_mask(const ImageDesc *desc_dev, int nimg, long long total_words,
                             const long long *img_word_begin_dev, const uint8_t *mask, uint32_t *bits,
                             cudaStream_t s);
constexpr int kMeanBlocks = 64;  // CTAs per plane in the observed-mean reduction
template <typename T>
cudaError_t launch_means(const ImageDesc *desc_dev, int nplanes, const int *plane_img_dev, const T *y,
                         const uint32_t *bits, double *partial, double *means, cudaStream_t s);
template <typename T>
cudaError_t launch_init_fill(const ImageDesc *desc_dev, int nimg, long long total_px,
                             const long long *img_px_begin_dev, const T *y, const uint32_t *bits,
                             const double *means, int K, T *yt, cudaStream_t s);
// Penalty adaptation (Eq. (varying_penalty)): per image, reduce the residual
// partials of ROW_NORMS and update mu, mu_prev and the d rescaling factor.
cudaError_t launch_mu_update(const ImageDesc *desc_dev, int nimg, const double *apart, double *mu, double *mu_prev,
                             double *dscale, double t, cudaStream_t s);
// mu = mu_prev = mu0, dscale = 1 for nimg images.
cudaError_t launch_mu_fill(double *mu, double *mu_prev, double *dscale, int nimg, double mu0, cudaStream_t s);
cudaError_t launch_stats_reduce(const ImageDesc *desc_dev, int nimg, const double *partials, double *stats,
                                int iters, int it, int *err, cudaStream_t s);

}  // namespace dcv
