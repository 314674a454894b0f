/*
 * FP64 CPU oracle for the partial-ADMM deconvolution with incomplete
 * observations (Simoes, Almeida, Bioucas-Dias, Chanussot, arXiv:1602.01410).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code with the
 * CUDA path: its convolutions are direct spatial sums, its DFT is its own
 * recursive mixed-radix transform, and its solve follows the paper's steps in
 * the paper's order.  It is deliberately plain and slow.
 *
 * Layout: images are row-major M x N doubles (M rows of the extended grid,
 * Sec. I-A); C channels are stacked [C][M][N] (Sec. III-C, demosaicing).  The
 * kernel h is (2b+1) x (2b+1) row-major with its origin at h[b][b].
 *
 * Parity status: every function here is pinned by the CPU test suite
 * (naive DFT and numpy.fft for the FFT, scipy convolution for the blurs,
 * adjoint identities, brute-force prox, normal equations, Lemma 3
 * monotonicity, the lambda = 0 closed form and a dense standard-ADMM run).
 * The gradient (reverse pass) is pinned by central finite differences of
 * the forward oracle: per parameter (lambda and every kernel tap) and along
 * random directions of (lambda, h), one and three channels, relax 1 and 2.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* ---------------------------------------------------------------- DFT ---
 * X[k] = sum_n x[n] exp(sign * 2 pi i n k / L).  Recursive decimation in time
 * on the smallest prime factor p of L: L = p m, the p interleaved
 * sub-sequences x[p j + r] are transformed (length m), then combined with
 * X[k + q m] = sum_r exp(sign 2 pi i r (k + q m) / L) Y_r[k].  Plain
 * textbook Cooley-Tukey; a prime length is a direct DFT.
 */
static int smallest_factor(int n) {
  for (int p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

/* Roots of unity of the top-level length L, tw[k] = exp(sign 2 pi i k / L),
 * from libm cos/sin in double; a sub-transform of length n uses
 * exp(sign 2 pi i idx / n) = tw[(idx mod n) * (L / n)]. */
typedef struct {
  int L;
  cplx *tw;
} roots;

static roots make_roots(int L, int sign) {
  roots r = {L, malloc(sizeof(cplx) * (size_t)L)};
  for (int k = 0; k < L; ++k) {
    double a = sign * 2.0 * M_PI * (double)k / (double)L;
    r.tw[k] = cos(a) + I * sin(a);
  }
  return r;
}

static void fft_rec(const cplx *in, int stride, cplx *out, int n, const roots *w, cplx *scratch) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  int p = smallest_factor(n);
  int m = n / p;
  int step = w->L / n;
  for (int r = 0; r < p; ++r) fft_rec(in + (size_t)r * stride, stride * p, out + (size_t)r * m, m, w, scratch);
  for (int q = 0; q < p; ++q)
    for (int k = 0; k < m; ++k) {
      cplx acc = 0;
      for (int r = 0; r < p; ++r) acc += out[(size_t)r * m + k] * w->tw[(size_t)((r * (k + q * m)) % n) * step];
      scratch[(size_t)q * m + k] = acc;
    }
  memcpy(out, scratch, sizeof(cplx) * (size_t)n);
}

/* In-place 1-D DFT of n interleaved (re, im) doubles; unnormalised. */
int or_fft1d(double *data, int n, int sign) {
  if (n <= 0) return -1;
  cplx *in = malloc(sizeof(cplx) * n), *out = malloc(sizeof(cplx) * n), *scr = malloc(sizeof(cplx) * n);
  roots w = make_roots(n, sign);
  for (int i = 0; i < n; ++i) in[i] = data[2 * i] + I * data[2 * i + 1];
  fft_rec(in, 1, out, n, &w, scr);
  free(w.tw);
  for (int i = 0; i < n; ++i) {
    data[2 * i] = creal(out[i]);
    data[2 * i + 1] = cimag(out[i]);
  }
  free(in); free(out); free(scr);
  return 0;
}

/* 2-D DFT of an M x N complex array: every row, then every column. */
static void fft2(cplx *a, int M, int N, int sign) {
  roots wr = make_roots(N, sign), wc = make_roots(M, sign);
#pragma omp parallel
  {
    int L = M > N ? M : N;
    cplx *in = malloc(sizeof(cplx) * L), *out = malloc(sizeof(cplx) * L), *scr = malloc(sizeof(cplx) * L);
#pragma omp for
    for (int i = 0; i < M; ++i) {
      fft_rec(a + (size_t)i * N, 1, out, N, &wr, scr);
      memcpy(a + (size_t)i * N, out, sizeof(cplx) * N);
    }
#pragma omp for
    for (int j = 0; j < N; ++j) {
      for (int i = 0; i < M; ++i) in[i] = a[(size_t)i * N + j];
      fft_rec(in, 1, out, M, &wc, scr);
      for (int i = 0; i < M; ++i) a[(size_t)i * N + j] = out[i];
    }
    free(in); free(out); free(scr);
  }
  free(wr.tw);
  free(wc.tw);
}

int or_fft2d(double *data, int M, int N, int sign) {
  size_t P = (size_t)M * N;
  cplx *a = malloc(sizeof(cplx) * P);
  for (size_t i = 0; i < P; ++i) a[i] = data[2 * i] + I * data[2 * i + 1];
  fft2(a, M, N, sign);
  for (size_t i = 0; i < P; ++i) {
    data[2 * i] = creal(a[i]);
    data[2 * i + 1] = cimag(a[i]);
  }
  free(a);
  return 0;
}

/* ------------------------------------------------------ blur operators ---
 * Eq. (4): T~ is the BCCB matrix of the circular convolution with h on the
 * M x N grid, (T~x)[i][j] = sum_{p,q=-b..b} h[p+b][q+b] x[(i-p)%M][(j-q)%N].
 * Eq. (1): T is the linear 'valid' convolution, defined on the central
 * (M-2b) x (N-2b) region.  Both are written as direct sums.
 */
static inline int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

/* Periodic extension of x by b pixels on every side: xp[i+b][j+b] = x[i%M][j%N]. */
static double *periodic_pad(const double *x, int M, int N, int b) {
  int W = N + 2 * b;
  double *xp = malloc(sizeof(double) * (size_t)(M + 2 * b) * W);
  for (int i = -b; i < M + b; ++i)
    for (int j = -b; j < N + b; ++j) xp[(size_t)(i + b) * W + (j + b)] = x[(size_t)wrap(i, M) * N + wrap(j, N)];
  return xp;
}

void or_conv_circ(const double *x, int M, int N, const double *h, int K, double *out) {
  int b = K / 2, W = N + 2 * b;
  double *xp = periodic_pad(x, M, N, b);
#pragma omp parallel for
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
      for (int p = -b; p <= b; ++p)
        for (int q = -b; q <= b; ++q) s += h[(p + b) * K + (q + b)] * xp[(size_t)(i - p + b) * W + (j - q + b)];
      out[(size_t)i * N + j] = s;
    }
  free(xp);
}

/* T~^T: circular correlation, (T~^T y)[i][j] = sum h[p+b][q+b] y[(i+p)%M][(j+q)%N]. */
void or_conv_circ_adj(const double *y, int M, int N, const double *h, int K, double *out) {
  int b = K / 2, W = N + 2 * b;
  double *yp = periodic_pad(y, M, N, b);
#pragma omp parallel for
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
      for (int p = -b; p <= b; ++p)
        for (int q = -b; q <= b; ++q) s += h[(p + b) * K + (q + b)] * yp[(size_t)(i + p + b) * W + (j + q + b)];
      out[(size_t)i * N + j] = s;
    }
  free(yp);
}

/* T x on the valid region: out[(i-b)][(j-b)] for i in [b, M-b), j in [b, N-b). */
void or_conv_valid(const double *x, int M, int N, const double *h, int K, double *out) {
  int b = K / 2, m = M - 2 * b, n = N - 2 * b;
#pragma omp parallel for
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int p = -b; p <= b; ++p)
        for (int q = -b; q <= b; ++q) s += h[(p + b) * K + (q + b)] * x[(size_t)(i + b - p) * N + (j + b - q)];
      out[(size_t)i * n + j] = s;
    }
}

/* -------------------------------------------------- first differences ---
 * Sec. III-B (isotropic TV): D_h, D_v are horizontal and vertical first-order
 * differences with periodic boundaries; here forward differences,
 * (D_h x)[i][j] = x[i][j+1] - x[i][j], (D_v x)[i][j] = x[i+1][j] - x[i][j].
 */
void or_diff_fwd(const double *x, int M, int N, double *dh, double *dv) {
#pragma omp parallel for
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      double c = x[(size_t)i * N + j];
      dh[(size_t)i * N + j] = x[(size_t)i * N + wrap(j + 1, N)] - c;
      dv[(size_t)i * N + j] = x[(size_t)wrap(i + 1, M) * N + j] - c;
    }
}

/* D^T [u_h; u_v] = D_h^T u_h + D_v^T u_v, the transpose of or_diff_fwd. */
void or_diff_adj(const double *uh, const double *uv, int M, int N, double *out) {
#pragma omp parallel for
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      size_t o = (size_t)i * N + j;
      out[o] = uh[(size_t)i * N + wrap(j - 1, N)] - uh[o] + uv[(size_t)wrap(i - 1, M) * N + j] - uv[o];
    }
}

/* ----------------------------------------------------- vector soft ---
 * Sec. III-B: the prox of tau * sum_j ||a_j|| (isotropic, or vectorial over
 * channels for Sec. III-C demosaicing) is the vector soft-threshold,
 * v_j = max(||a_j|| - tau, 0) a_j / ||a_j||, v_j = 0 when ||a_j|| <= tau.
 * a is laid out as `dim` planes of n values; the norm at pixel j runs over the
 * planes.
 */
void or_vsoft(const double *a, int n, int dim, double tau, double *v) {
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int c = 0; c < dim; ++c) s += a[(size_t)c * n + j] * a[(size_t)c * n + j];
    double nrm = sqrt(s);
    double g = nrm > tau ? (nrm - tau) / nrm : 0.0;
    for (int c = 0; c < dim; ++c) v[(size_t)c * n + j] = g * a[(size_t)c * n + j];
  }
}

/* ------------------------------------------------------- x-step solve ---
 * Eq. (dual_x_iter_resolved_boundaries): x = (H^T H + mu D^T D)^{-1} rhs with
 * H^T H = T~^T T~ (BCCB) and D^T D BCCB; the paper solves it in the DFT
 * domain.  The eigenvalues of the BCCB matrix A = T~^T T~ + mu D^T D are the
 * DFT of its first column, A e_0, which is computed here with the spatial
 * operators above: den = DFT2(A e_0).
 */
static double *solve_denominator(int M, int N, const double *h, int K, double mu) {
  size_t P = (size_t)M * N;
  double *e = calloc(P, sizeof(double)), *t = malloc(P * sizeof(double)), *a = malloc(P * sizeof(double));
  double *uh = malloc(P * sizeof(double)), *uv = malloc(P * sizeof(double)), *dd = malloc(P * sizeof(double));
  e[0] = 1.0;
  or_conv_circ(e, M, N, h, K, t);
  or_conv_circ_adj(t, M, N, h, K, a);
  or_diff_fwd(e, M, N, uh, uv);
  or_diff_adj(uh, uv, M, N, dd);
  cplx *s = malloc(sizeof(cplx) * P);
  for (size_t i = 0; i < P; ++i) s[i] = a[i] + mu * dd[i];
  fft2(s, M, N, -1);
  double *den = malloc(P * sizeof(double));
  for (size_t i = 0; i < P; ++i) den[i] = creal(s[i]); /* A is symmetric: real spectrum */
  free(e); free(t); free(a); free(uh); free(uv); free(dd); free(s);
  return den;
}

static void solve_x(const double *rhs, const double *den, int M, int N, double *x, cplx *work) {
  size_t P = (size_t)M * N;
  for (size_t i = 0; i < P; ++i) work[i] = rhs[i];
  fft2(work, M, N, -1);
  for (size_t i = 0; i < P; ++i) work[i] /= den[i];
  fft2(work, M, N, +1);
  for (size_t i = 0; i < P; ++i) x[i] = creal(work[i]) / (double)P;
}

/* Public wrapper for tests: x = (T~^T T~ + mu D^T D)^{-1} rhs. */
void or_solve_x(const double *rhs, int M, int N, const double *h, int K, double mu, double *x) {
  double *den = solve_denominator(M, N, h, K, mu);
  cplx *w = malloc(sizeof(cplx) * (size_t)M * N);
  solve_x(rhs, den, M, N, x, w);
  free(den); free(w);
}

/* ------------------------------------------------------ initial state ---
 * Sec. III-B: x is initialised by padding the observed image with its
 * border pixels.  Reading used here (the paper is silent on interior holes):
 * an unobserved pixel of the boundary band takes the value at the clamped
 * valid-region index when that pixel is observed; every other unobserved
 * pixel takes the mean of the observed values of its channel (computed in
 * double, then rounded once with `round_f32`).  y~0 is that padded image.
 */
void or_init_ytilde(const double *y, const uint8_t *mask, int M, int N, int K, int round_f32, double *yt) {
  int b = K / 2;
  double s = 0.0;
  long cnt = 0;
  for (size_t i = 0; i < (size_t)M * N; ++i)
    if (mask[i]) {
      s += y[i];
      ++cnt;
    }
  double mean = cnt ? s / (double)cnt : 0.0;
  if (round_f32) mean = (double)(float)mean;
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      size_t o = (size_t)i * N + j;
      if (mask[o]) {
        yt[o] = y[o];
        continue;
      }
      int band = (i < b || i >= M - b || j < b || j >= N - b);
      double v = mean;
      if (band) {
        int ic = i < b ? b : (i >= M - b ? M - b - 1 : i);
        int jc = j < b ? b : (j >= N - b ? N - b - 1 : j);
        size_t oc = (size_t)ic * N + jc;
        if (mask[oc]) v = y[oc];
      }
      yt[o] = v;
    }
}

/* ------------------------------------------- Tikhonov initialisation ---
 * Sec. III-B, Eqs. (ini_x)-(ini_z): z is initialised by alternating
 * minimisation of f(x, z) + tau/2 ||x||^2,
 *   x^i = (H^T H + tau I)^{-1} H^T [y; z^{i-1}],   z^i = M_z H x^i,
 * from z^0 = the padded observation (yt on entry).  H^T H + tau I is BCCB;
 * its eigenvalues are the DFT of its first column (T~^T T~ e_0 + tau e_0).
 * One channel plane; yt is updated in place (unobserved entries), x
 * receives x^{iters}.
 */
static double *tikhonov_denominator(int M, int N, const double *h, int K, double tau) {
  size_t P = (size_t)M * N;
  double *e = calloc(P, sizeof(double)), *t = malloc(P * sizeof(double)), *a = malloc(P * sizeof(double));
  e[0] = 1.0;
  or_conv_circ(e, M, N, h, K, t);
  or_conv_circ_adj(t, M, N, h, K, a);
  cplx *s = malloc(sizeof(cplx) * P);
  for (size_t i = 0; i < P; ++i) s[i] = a[i] + tau * e[i];
  fft2(s, M, N, -1);
  double *den = malloc(P * sizeof(double));
  for (size_t i = 0; i < P; ++i) den[i] = creal(s[i]);
  free(e); free(t); free(a); free(s);
  return den;
}

void or_tikhonov(int M, int N, int K, const double *h, const uint8_t *mask, int iters, double tau, double *yt,
                 double *x) {
  size_t P = (size_t)M * N;
  double *den = tikhonov_denominator(M, N, h, K, tau);
  double *rhs = malloc(P * sizeof(double)), *tmp = malloc(P * sizeof(double));
  cplx *work = malloc(sizeof(cplx) * P);
  for (int it = 0; it < iters; ++it) {
    or_conv_circ_adj(yt, M, N, h, K, rhs); /* H^T [y; z] = T~^T y~ */
    solve_x(rhs, den, M, N, x, work);
    or_conv_circ(x, M, N, h, K, tmp);
    for (size_t i = 0; i < P; ++i)
      if (!mask[i]) yt[i] = tmp[i]; /* z = M_z H x */
  }
  free(den); free(rhs); free(tmp); free(work);
}

/* ------------------------------------------------------ partial ADMM ---
 * Eqs. (admm_aprox_1)-(admm_aprox_4), the closed forms
 * (dual_x_iter_resolved_boundaries) for x and the over-relaxed z-update
 * z = relax * M_z H x - (relax - 1) z (relax = 2 in Sec. II-B, relax = 1 is
 * the plain Eq. (dual_z_iter_resolved_boundaries)).  C channels share the
 * blur; the TV norm couples them (vectorial TV, Sec. III-C).
 *
 * passes >= 1: block-Gauss-Seidel passes of steps (admm_aprox_1)-(admm_aprox_2)
 * per iteration (Sec. II-C: an inner loop on x and z with v and d fixed;
 * "Proposed-AD" uses b passes for a (2b+1) x (2b+1) blur, Sec. III-B).
 * adapt_t > 0: penalty adaptation of Eq. (varying_penalty) after every
 * iteration with threshold t: mu doubles (d halves) when
 * ||d^{i+1} - d^i|| > t ||v^{i+1} - v^i||, mu halves (d doubles) when
 * ||v^{i+1} - v^i|| > t ||d^{i+1} - d^i||; norms over all channels of the
 * image.  tikh_iters > 0 (init only): Tikhonov warm start of z (or_tikhonov
 * per channel, tau = tikh_tau), then x^0 = its last x.
 *
 * State (in/out when init == 0, out when init == 1): yt = y~ (observed
 * entries hold y, unobserved hold z), d = d_x as [C][2][M][N] (h then v
 * component), v = v_x with the same layout; *mu_io = mu in, the final mu out.
 * Initial state (init == 1): y~^0 = or_init_ytilde (then the warm start, if
 * any), d^0 = 0, v^0 = D x^0 with x^0 = y~^0, or the warm start's x.
 * Output x = x^{iters} (x^0 when iters = 0 from the initial state).  stats (nullable) receives per iteration
 *   [ ||d^{i+1}-d^i||^2, ||z^{i+1}-z^i||^2, mu ||v^{i+1}-v^i||^2, J(x^{i+1}) ]
 * (z change and x of the last pass; d^{i+1} before the rescaling; mu = mu^i)
 * with J(x) = 1/2 sum_obs (y - T~x)^2 + lambda sum_j ||(Dx)_j||, the
 * objective of Eq. (problem_xz) minimised over z.  mu_hist (nullable)
 * receives mu^i, the penalty each iteration used.
 */
int or_admm_ex(int C, int M, int N, int K, const double *h, const double *y, const uint8_t *mask,
               double lambda, double *mu_io, double relax, int iters, int init, int round_f32, int passes,
               double adapt_t, int tikh_iters, double tikh_tau, double *yt, double *d, double *v, double *x,
               double *stats, double *mu_hist) {
  size_t P = (size_t)M * N;
  double mu = *mu_io;
  if (passes < 1) return 1;
  double *den = solve_denominator(M, N, h, K, mu);
  double *rhs = malloc(P * sizeof(double)), *tmp = malloc(P * sizeof(double));
  double *dx = malloc(2 * C * P * sizeof(double)), *a = malloc(2 * C * P * sizeof(double));
  double *vn = malloc(2 * C * P * sizeof(double));
  cplx *work = malloc(sizeof(cplx) * P);

  if (init) {
    for (int c = 0; c < C; ++c) {
      or_init_ytilde(y + c * P, mask + c * P, M, N, K, round_f32, yt + c * P);
      if (tikh_iters > 0) {
        or_tikhonov(M, N, K, h, mask + c * P, tikh_iters, tikh_tau, yt + c * P, x + c * P);
        or_diff_fwd(x + c * P, M, N, v + 2 * c * P, v + (2 * c + 1) * P); /* v0 = D x0, x0 = warm-start x */
      } else {
        memcpy(x + c * P, yt + c * P, P * sizeof(double));                  /* x0 = y~0 */
        or_diff_fwd(yt + c * P, M, N, v + 2 * c * P, v + (2 * c + 1) * P); /* v0 = D x0 */
      }
    }
    memset(d, 0, 2 * C * P * sizeof(double));
  }
  for (int it = 0; it < iters; ++it) {
    if (mu_hist) mu_hist[it] = mu;
    double dz2 = 0.0;
    for (int pass = 0; pass < passes; ++pass) {
      /* (admm_aprox_1): x = (H^T H + mu D^T D)^{-1} [H^T [y; z] + mu D^T (v - d)] */
      for (int c = 0; c < C; ++c) {
        double *uh = a + 2 * c * P, *uv = a + (2 * c + 1) * P;
        for (size_t i = 0; i < P; ++i) {
          uh[i] = v[2 * c * P + i] - d[2 * c * P + i];
          uv[i] = v[(2 * c + 1) * P + i] - d[(2 * c + 1) * P + i];
        }
        or_diff_adj(uh, uv, M, N, tmp);
        or_conv_circ_adj(yt + c * P, M, N, h, K, rhs);
        for (size_t i = 0; i < P; ++i) rhs[i] += mu * tmp[i];
        solve_x(rhs, den, M, N, x + c * P, work);
      }
      /* (admm_aprox_2), over-relaxed: z = relax M_z H x - (relax - 1) z */
      dz2 = 0.0;
      for (int c = 0; c < C; ++c) {
        or_conv_circ(x + c * P, M, N, h, K, tmp);
        for (size_t i = 0; i < P; ++i)
          if (!mask[c * P + i]) {
            double zn = relax * tmp[i] - (relax - 1.0) * yt[c * P + i];
            dz2 += (zn - yt[c * P + i]) * (zn - yt[c * P + i]);
            yt[c * P + i] = zn;
          }
      }
    }
    /* (admm_aprox_3): v = vector-soft(D x + d, lambda / mu) */
    for (int c = 0; c < C; ++c) or_diff_fwd(x + c * P, M, N, dx + 2 * c * P, dx + (2 * c + 1) * P);
    for (size_t i = 0; i < 2 * C * P; ++i) a[i] = dx[i] + d[i];
    or_vsoft(a, (int)P, 2 * C, lambda / mu, vn);
    /* (admm_aprox_4): d = d - (v - D x) = a - v */
    double dd2 = 0.0, dv2 = 0.0;
    for (size_t i = 0; i < 2 * C * P; ++i) {
      double dn = a[i] - vn[i];
      dd2 += (dn - d[i]) * (dn - d[i]);
      dv2 += (vn[i] - v[i]) * (vn[i] - v[i]);
      d[i] = dn;
      v[i] = vn[i];
    }
    if (stats) {
      double fit = 0.0, tv = 0.0;
      for (int c = 0; c < C; ++c) {
        or_conv_circ(x + c * P, M, N, h, K, tmp);
        for (size_t i = 0; i < P; ++i)
          if (mask[c * P + i]) fit += (y[c * P + i] - tmp[i]) * (y[c * P + i] - tmp[i]);
      }
      for (size_t i = 0; i < P; ++i) {
        double s = 0.0;
        for (int k = 0; k < 2 * C; ++k) s += dx[k * P + i] * dx[k * P + i];
        tv += sqrt(s);
      }
      stats[4 * it + 0] = dd2;
      stats[4 * it + 1] = dz2;
      stats[4 * it + 2] = mu * dv2;
      stats[4 * it + 3] = 0.5 * fit + lambda * tv;
    }
    /* Eq. (varying_penalty) and the rescaling of d */
    if (adapt_t > 0.0) {
      double nd = sqrt(dd2), nv = sqrt(dv2), f = 1.0;
      if (nd > adapt_t * nv) f = 2.0;
      else if (nv > adapt_t * nd) f = 0.5;
      if (f != 1.0) {
        mu *= f;
        for (size_t i = 0; i < 2 * C * P; ++i) d[i] /= f;
        free(den);
        den = solve_denominator(M, N, h, K, mu);
      }
    }
  }
  *mu_io = mu;
  free(den); free(rhs); free(tmp); free(dx); free(a); free(vn); free(work);
  return 0;
}

/* One BGS pass, fixed mu, no warm start (the iteration the paper calls
 * Proposed-1). */
int or_admm(int C, int M, int N, int K, const double *h, const double *y, const uint8_t *mask,
            double lambda, double mu, double relax, int iters, int init, int round_f32,
            double *yt, double *d, double *v, double *x, double *stats) {
  return or_admm_ex(C, M, N, K, h, y, mask, lambda, &mu, relax, iters, init, round_f32, 1, 0.0, 0, 0.0, yt, d, v, x,
                    stats, NULL);
}

/* --------------------------------------------------- reverse pass (grad) ---
 * Gradient of L = mean over all C*M*N pixels of (x^{iters} - x_true)^2 with
 * respect to lambda and the kernel taps h, through `iters` iterations of
 * or_admm (from the initial fill, relax as given).  Reverse-mode
 * differentiation of the steps of Eqs. (admm_aprox_1)-(admm_aprox_4) as
 * written above, in reverse order; every forward quantity is stored (this is
 * a small-size reference, not a checkpointed implementation).
 * Per step i (a = D x^{i+1} + d^i, adjoints carried: yb, vb, db):
 *   w = vb - db;  ab = db + J(a) w   (J the Jacobian of vector-soft, Sec. III-B)
 *   taub -= sum_j a_j^T w_j / ||a_j||  over pixels with ||a_j|| > tau
 *   tb = relax M_u yb;  yb' = (M_o - (relax-1) M_u) yb;  xb = D^T ab (+ dL/dx)
 *   bb = (T~^T T~ + mu D^T D)^{-1} (xb + T~^T tb)
 *   hb += corr(bb, y~^i - T~x^{i+1}) + corr(x^{i+1}, tb - T~ bb)
 *   yb = yb' + T~ bb;  vb = mu D bb;  db = ab - mu D bb
 * with corr(u, w)[m] = sum_n u[n - m] w[n] at the kernel offsets m.
 * dlambda = taub / mu (tau = lambda / mu).  dh is K*K, row-major like h.
 */
static void corr_taps(const double *u, const double *w, int M, int N, int K, double *acc) {
  int b = K / 2;
  for (int p = -b; p <= b; ++p)
    for (int q = -b; q <= b; ++q) {
      double s = 0.0;
#pragma omp parallel for reduction(+ : s)
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < N; ++j) s += u[(size_t)wrap(i - p, M) * N + wrap(j - q, N)] * w[(size_t)i * N + j];
      acc[(p + b) * K + (q + b)] += s;
    }
}

int or_admm_grad(int C, int M, int N, int K, const double *h, const double *y, const uint8_t *mask, double lambda,
                 double mu, double relax, int iters, int round_f32, const double *x_true, double *loss,
                 double *dlambda, double *dh, double *x_out) {
  size_t P = (size_t)M * N, CP = (size_t)C * P;
  double tau = lambda / mu;
  double *den = solve_denominator(M, N, h, K, mu);
  cplx *work = malloc(sizeof(cplx) * P);
  /* stored forward quantities */
  double *YT = malloc(sizeof(double) * CP * (iters + 1));       /* y~^i */
  double *X = malloc(sizeof(double) * CP * (iters + 1));        /* x^i (x^0 unused) */
  double *TX = malloc(sizeof(double) * CP * (iters + 1));       /* T~ x^i */
  double *A = malloc(sizeof(double) * 2 * CP * (iters + 1));    /* a^i = D x^i + d^{i-1} */
  double *v = malloc(sizeof(double) * 2 * CP), *d = malloc(sizeof(double) * 2 * CP);
  double *rhs = malloc(sizeof(double) * P), *tmp = malloc(sizeof(double) * P), *tmp2 = malloc(sizeof(double) * P);
  double *dx = malloc(sizeof(double) * 2 * CP);
  for (int c = 0; c < C; ++c) {
    or_init_ytilde(y + c * P, mask + c * P, M, N, K, round_f32, YT + c * P);
    or_diff_fwd(YT + c * P, M, N, v + 2 * c * P, v + (2 * c + 1) * P);
  }
  memset(d, 0, sizeof(double) * 2 * CP);
  for (int it = 0; it < iters; ++it) {
    double *yt = YT + CP * it, *ytn = YT + CP * (it + 1), *x = X + CP * (it + 1), *tx = TX + CP * (it + 1);
    double *a = A + 2 * CP * (it + 1);
    for (int c = 0; c < C; ++c) {
      for (size_t i = 0; i < P; ++i) {
        tmp[i] = v[2 * c * P + i] - d[2 * c * P + i];
        tmp2[i] = v[(2 * c + 1) * P + i] - d[(2 * c + 1) * P + i];
      }
      or_diff_adj(tmp, tmp2, M, N, rhs);
      for (size_t i = 0; i < P; ++i) rhs[i] *= mu;
      or_conv_circ_adj(yt + c * P, M, N, h, K, tmp);
      for (size_t i = 0; i < P; ++i) rhs[i] += tmp[i];
      solve_x(rhs, den, M, N, x + c * P, work);
      or_conv_circ(x + c * P, M, N, h, K, tx + c * P);
      for (size_t i = 0; i < P; ++i)
        ytn[c * P + i] = mask[c * P + i] ? yt[c * P + i] : relax * tx[c * P + i] - (relax - 1.0) * yt[c * P + i];
      or_diff_fwd(x + c * P, M, N, dx + 2 * c * P, dx + (2 * c + 1) * P);
    }
    for (size_t i = 0; i < 2 * CP; ++i) a[i] = dx[i] + d[i];
    or_vsoft(a, (int)P, 2 * C, tau, v);
    for (size_t i = 0; i < 2 * CP; ++i) d[i] = a[i] - v[i];
  }
  double *xK = X + CP * iters;
  double cnt = (double)CP, L = 0.0;
  for (size_t i = 0; i < CP; ++i) L += (xK[i] - x_true[i]) * (xK[i] - x_true[i]);
  *loss = L / cnt;
  if (x_out) memcpy(x_out, xK, sizeof(double) * CP);

  double *yb = calloc(CP, sizeof(double)), *vb = calloc(2 * CP, sizeof(double)), *db = calloc(2 * CP, sizeof(double));
  double *ab = malloc(sizeof(double) * 2 * CP), *wv = malloc(sizeof(double) * 2 * CP);
  double *xb = malloc(sizeof(double) * CP), *tb = malloc(sizeof(double) * CP), *bb = malloc(sizeof(double) * CP);
  double *tbb = malloc(sizeof(double) * CP), *e = malloc(sizeof(double) * P);
  double taub = 0.0;
  for (int t = 0; t < K * K; ++t) dh[t] = 0.0;
  for (int it = iters - 1; it >= 0; --it) {
    double *a = A + 2 * CP * (it + 1), *x = X + CP * (it + 1), *tx = TX + CP * (it + 1), *yt = YT + CP * it;
    for (size_t i = 0; i < 2 * CP; ++i) wv[i] = vb[i] - db[i];
    for (size_t j = 0; j < P; ++j) {
      double n2 = 0.0, aw = 0.0;
      for (int k = 0; k < 2 * C; ++k) {
        n2 += a[k * P + j] * a[k * P + j];
        aw += a[k * P + j] * wv[k * P + j];
      }
      double n = sqrt(n2);
      for (int k = 0; k < 2 * C; ++k) {
        double g = 0.0;
        if (n > tau) g = (1.0 - tau / n) * wv[k * P + j] + tau * a[k * P + j] * aw / (n2 * n);
        ab[k * P + j] = db[k * P + j] + g;
      }
      if (n > tau) taub -= aw / n;
    }
    for (int c = 0; c < C; ++c) {
      for (size_t i = 0; i < P; ++i) {
        double yv = yb[c * P + i];
        int obs = mask[c * P + i] != 0;
        tb[c * P + i] = obs ? 0.0 : relax * yv;
        yb[c * P + i] = obs ? yv : -(relax - 1.0) * yv; /* yb' */
      }
      or_diff_adj(ab + 2 * c * P, ab + (2 * c + 1) * P, M, N, xb + c * P);
      if (it == iters - 1)
        for (size_t i = 0; i < P; ++i) xb[c * P + i] += 2.0 * (xK[c * P + i] - x_true[c * P + i]) / cnt;
      or_conv_circ_adj(tb + c * P, M, N, h, K, rhs);
      for (size_t i = 0; i < P; ++i) rhs[i] += xb[c * P + i];
      solve_x(rhs, den, M, N, bb + c * P, work);
      or_conv_circ(bb + c * P, M, N, h, K, tbb + c * P);
      for (size_t i = 0; i < P; ++i) e[i] = yt[c * P + i] - tx[c * P + i];
      corr_taps(bb + c * P, e, M, N, K, dh);
      for (size_t i = 0; i < P; ++i) e[i] = tb[c * P + i] - tbb[c * P + i];
      corr_taps(x + c * P, e, M, N, K, dh);
      for (size_t i = 0; i < P; ++i) yb[c * P + i] += tbb[c * P + i];
      or_diff_fwd(bb + c * P, M, N, tmp, tmp2);
      for (size_t i = 0; i < P; ++i) {
        vb[2 * c * P + i] = mu * tmp[i];
        vb[(2 * c + 1) * P + i] = mu * tmp2[i];
        db[2 * c * P + i] = ab[2 * c * P + i] - mu * tmp[i];
        db[(2 * c + 1) * P + i] = ab[(2 * c + 1) * P + i] - mu * tmp2[i];
      }
    }
  }
  *dlambda = taub / mu;
  free(den); free(work); free(YT); free(X); free(TX); free(A); free(v); free(d); free(rhs); free(tmp); free(tmp2);
  free(dx); free(yb); free(vb); free(db); free(ab); free(wv); free(xb); free(tb); free(bb); free(tbb); free(e);
  return 0;
}
