// One-time and per-solve setup kernels.
#include "fft.cuh"
#include "internal.h"

namespace dcv {

// H^(k1, k2) = sum_{p,q=-b..b} h[p+b][q+b] exp(-2 pi i (k1 p / M + k2 q / N)),
// the DFT of the kernel placed with its origin at grid index (0, 0) (the
// eigenvalues of the BCCB matrix T~ of Eq. (4)), in double precision and
// separably: first the K x (N/2+1) row sums
//   G(p, k2) = sum_q h[p+b][q+b] exp(-2 pi i k2 q / N),
// then H^(k1, k2) = sum_p G(p, k2) exp(-2 pi i k1 p / M), rounded once to T.
// In each sum the phase of the first tap is reduced exactly in integers and
// the following taps' twiddles come from multiplying by exp(-2 pi i k / L)
// (about (2b+1) ulp of drift in double).
__device__ __forceinline__ void root_pi(long long k, long long n, long long L, double *c, double *s) {
  const long long ph = (((k * n) % L) + L) % L;
  sincospi(-2.0 * (double)ph / (double)L, s, c);
}

__device__ __forceinline__ int find_job(const long long *begin, int njobs, long long e) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void hrow_kernel(const HhatJob *jobs, int njobs, const long long *g_begin, long long total, const T *h,
                            double2 *G) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int j = find_job(g_begin, njobs, e);
  const HhatJob J = jobs[j];
  const long long loc = e - g_begin[j];
  const int p = (int)(loc / J.Nh), k2 = (int)(loc - (long long)p * J.Nh);
  const int b = J.K / 2;
  double c, s, cs, ss;
  root_pi(k2, -b, J.N, &c, &s);
  root_pi(k2, 1, J.N, &cs, &ss);
  double re = 0.0, im = 0.0;
  for (int q = 0; q < J.K; ++q) {
    const double hv = (double)h[J.h + (long long)p * J.K + q];
    re += hv * c;
    im += hv * s;
    const double cn = c * cs - s * ss;
    s = c * ss + s * cs;
    c = cn;
  }
  G[J.g + loc] = make_double2(re, im);
}

template <typename T>
__global__ void hcol_kernel(const HhatJob *jobs, int njobs, const long long *job_begin, long long total,
                            const double2 *G, cx<T> *hhat) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int j = find_job(job_begin, njobs, e);
  const HhatJob J = jobs[j];
  const long long loc = e - job_begin[j];
  const int k1 = (int)(loc / J.Nh), k2 = (int)(loc - (long long)k1 * J.Nh);
  const int b = J.K / 2;
  double c, s, cs, ss;
  root_pi(k1, -b, J.M, &c, &s);
  root_pi(k1, 1, J.M, &cs, &ss);
  double re = 0.0, im = 0.0;
  const double2 *g = G + J.g + k2;
  for (int p = 0; p < J.K; ++p) {
    const double2 v = g[(long long)p * J.Nh];
    re += v.x * c - v.y * s;
    im += v.x * s + v.y * c;
    const double cn = c * cs - s * ss;
    s = c * ss + s * cs;
    c = cn;
  }
  hhat[J.out + loc] = mk<T>((T)re, (T)im);
}

template <typename T>
cudaError_t launch_hhat(const HhatJob *jobs_dev, int njobs, long long total, const T *h, void *hhat,
                        const long long *job_begin_dev, const long long *g_begin_dev, long long total_g, void *G,
                        cudaStream_t s) {
  const int nt = 256;
  hrow_kernel<T><<<(unsigned)((total_g + nt - 1) / nt), nt, 0, s>>>(jobs_dev, njobs, g_begin_dev, total_g, h,
                                                                     static_cast<double2 *>(G));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hcol_kernel<T><<<(unsigned)((total + nt - 1) / nt), nt, 0, s>>>(jobs_dev, njobs, job_begin_dev, total,
                                                                  static_cast<const double2 *>(G),
                                                                  reinterpret_cast<cx<T> *>(hhat));
  return cudaGetLastError();
}
template cudaError_t launch_hhat<float>(const HhatJob *, int, long long, const float *, void *, const long long *,
                                        const long long *, long long, void *, cudaStream_t);
template cudaError_t launch_hhat<double>(const HhatJob *, int, long long, const double *, void *,
                                         const long long *, const long long *, long long, void *, cudaStream_t);

// Packs the byte mask (nonzero = observed) into 32-bit words, one bit per
// pixel, each channel plane padded to whole words.
__global__ void pack_mask_kernel(const ImageDesc *desc, int nimg, const long long *img_word_begin,
                                 long long total_words, const uint8_t *mask, uint32_t *bits) {
  const long long wd = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (wd >= total_words) return;
  int lo = 0, hi = nimg - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (img_word_begin[mid] <= wd) lo = mid; else hi = mid - 1;
  }
  const ImageDesc &D = desc[lo];
  const long long loc = wd - img_word_begin[lo];
  const long long ch = loc / D.mask_plane, w = loc - ch * D.mask_plane;
  const long long P = (long long)D.M * D.N;
  const uint8_t *src = mask + D.px + ch * P;
  uint32_t v = 0;
  for (int b = 0; b < 32; ++b) {
    const long long p = w * 32 + b;
    if (p < P && src[p] != 0) v |= 1u << b;
  }
  bits[D.mask + loc] = v;
}

cudaError_t launch_pack_mask(const ImageDesc *desc_dev, int nimg, long long total_words,
                             const long long *img_word_begin_dev, const uint8_t *mask, uint32_t *bits,
                             cudaStream_t s) {
  const int nt = 256;
  pack_mask_kernel<<<(unsigned)((total_words + nt - 1) / nt), nt, 0, s>>>(desc_dev, nimg, img_word_begin_dev,
                                                                         total_words, mask, bits);
  return cudaGetLastError();
}

// Mean of the observed values of each (image, channel) plane, in double.
// kMeanBlocks CTAs per plane write partial (sum, count) pairs; one CTA per
// plane then adds them in a fixed order.
template <typename T>
__global__ void means_partial_kernel(const ImageDesc *desc, const int *plane_img, const T *y, const uint32_t *bits,
                                     double *partial) {
  const int plane = blockIdx.x / kMeanBlocks, part = blockIdx.x % kMeanBlocks;
  const int img = plane_img[2 * plane], ch = plane_img[2 * plane + 1];
  const ImageDesc &D = desc[img];
  const long long P = (long long)D.M * D.N;
  const T *src = y + D.px + ch * P;
  const long long w0 = D.mask + ch * D.mask_plane;
  double s = 0.0;
  long long c = 0;
  for (long long p = (long long)part * blockDim.x + threadIdx.x; p < P; p += (long long)kMeanBlocks * blockDim.x)
    if ((bits[w0 + (p >> 5)] >> (p & 31)) & 1u) {
      s += (double)src[p];
      ++c;
    }
  __shared__ double rs[256];
  __shared__ long long rc[256];
  rs[threadIdx.x] = s;
  rc[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rs[threadIdx.x] += rs[threadIdx.x + o];
      rc[threadIdx.x] += rc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * (long long)blockIdx.x] = rs[0];
    partial[2 * (long long)blockIdx.x + 1] = (double)rc[0];
  }
}

__global__ void means_final_kernel(const double *partial, int nplanes, double *means) {
  const int plane = blockIdx.x * blockDim.x + threadIdx.x;
  if (plane >= nplanes) return;
  double s = 0.0, c = 0.0;
  for (int k = 0; k < kMeanBlocks; ++k) {
    s += partial[2 * ((long long)plane * kMeanBlocks + k)];
    c += partial[2 * ((long long)plane * kMeanBlocks + k) + 1];
  }
  means[plane] = c > 0 ? s / c : 0.0;
}

template <typename T>
cudaError_t launch_means(const ImageDesc *desc_dev, int nplanes, const int *plane_img_dev, const T *y,
                         const uint32_t *bits, double *partial, double *means, cudaStream_t s) {
  means_partial_kernel<T><<<nplanes * kMeanBlocks, 256, 0, s>>>(desc_dev, plane_img_dev, y, bits, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  means_final_kernel<<<(nplanes + 127) / 128, 128, 0, s>>>(partial, nplanes, means);
  return cudaGetLastError();
}
template cudaError_t launch_means<float>(const ImageDesc *, int, const int *, const float *, const uint32_t *,
                                         double *, double *, cudaStream_t);
template cudaError_t launch_means<double>(const ImageDesc *, int, const int *, const double *, const uint32_t *,
                                          double *, double *, cudaStream_t);

// y~0 (Sec. III-B: the observed image padded by repeating its border
// pixels).  Observed pixels take y.  An unobserved pixel of the boundary band
// takes y at the clamped valid-region index when that pixel is observed;
// every other unobserved pixel takes the plane's observed mean rounded to T.
// y may alias yt (observed entries are then left untouched).
template <typename T>
__global__ void init_fill_kernel(const ImageDesc *desc, int nimg, const long long *img_px_begin, long long total,
                                 const T *y, const uint32_t *bits, const double *means, int K, T *yt) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= total) return;
  int lo = 0, hi = nimg - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (img_px_begin[mid] <= e) lo = mid; else hi = mid - 1;
  }
  const ImageDesc &D = desc[lo];
  const long long P = (long long)D.M * D.N, loc = e - D.px;
  const int ch = (int)(loc / P);
  const long long p = loc - ch * P;
  const int i = (int)(p / D.N), j = (int)(p - (long long)i * D.N);
  const long long w0 = D.mask + ch * D.mask_plane;
  const bool obs = (bits[w0 + (p >> 5)] >> (p & 31)) & 1u;
  if (obs) {
    if (y != yt) yt[e] = y[e];
    return;
  }
  const int b = D.kb;  // the image's own half support (K / 2 unless supports differ)
  T v = (T)means[(long long)lo * D.C + ch];  // every image of a plan has the same channel count
  const bool band = i < b || i >= D.M - b || j < b || j >= D.N - b;
  if (band) {
    const int ic = i < b ? b : (i >= D.M - b ? D.M - b - 1 : i);
    const int jc = j < b ? b : (j >= D.N - b ? D.N - b - 1 : j);
    const long long pc = (long long)ic * D.N + jc;
    if ((bits[w0 + (pc >> 5)] >> (pc & 31)) & 1u) v = y[D.px + ch * P + pc];
  }
  yt[e] = v;
}

template <typename T>
cudaError_t launch_init_fill(const ImageDesc *desc_dev, int nimg, long long total_px,
                             const long long *img_px_begin_dev, const T *y, const uint32_t *bits,
                             const double *means, int K, T *yt, cudaStream_t s) {
  const int nt = 256;
  init_fill_kernel<T><<<(unsigned)((total_px + nt - 1) / nt), nt, 0, s>>>(desc_dev, nimg, img_px_begin_dev,
                                                                          total_px, y, bits, means, K, yt);
  return cudaGetLastError();
}
template cudaError_t launch_init_fill<float>(const ImageDesc *, int, long long, const long long *, const float *,
                                             const uint32_t *, const double *, int, float *, cudaStream_t);
template cudaError_t launch_init_fill<double>(const ImageDesc *, int, long long, const long long *,
                                              const double *, const uint32_t *, const double *, int, double *,
                                              cudaStream_t);

// Per-image sums of the row-pass partials in a fixed order:
// stats[img][it][0..2] = ||d^{i+1} - d^i||^2, ||z^{i+1} - z^i||^2, J(x^{i+1}).
__global__ void stats_reduce_kernel(const ImageDesc *desc, const double *partials, double *stats, int iters,
                                    int it, int *err) {
  const int img = blockIdx.x;
  const ImageDesc &D = desc[img];
  __shared__ double r[3][128];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int q = threadIdx.x; q < D.row_blocks; q += blockDim.x) {
    const long long o = 3LL * (D.row_pbase + q);
    a += partials[o];
    b += partials[o + 1];
    c += partials[o + 2];
  }
  r[0][threadIdx.x] = a;
  r[1][threadIdx.x] = b;
  r[2][threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 3; ++k) r[k][threadIdx.x] += r[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double *out = stats + 3LL * ((long long)img * iters + it);
    out[0] = r[0][0];
    out[1] = r[1][0];
    out[2] = r[2][0];
    if (!isfinite(r[2][0])) atomicOr(err, 1);
  }
}

// One CTA per image: fixed-order FP64 reduction of the image's row-block
// partials, then the rule of Eq. (varying_penalty) with threshold t.
__global__ void mu_update_kernel(const ImageDesc *desc, const double *apart, double *mu, double *mu_prev,
                                 double *dscale, double t) {
  const int img = blockIdx.x;
  const ImageDesc &D = desc[img];
  __shared__ double r[2][128];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < D.row_blocks; q += blockDim.x) {
    a += apart[2LL * (D.row_pbase + q)];
    b += apart[2LL * (D.row_pbase + q) + 1];
  }
  r[0][threadIdx.x] = a;
  r[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      r[0][threadIdx.x] += r[0][threadIdx.x + o];
      r[1][threadIdx.x] += r[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nd = sqrt(r[0][0]), nv = sqrt(r[1][0]);
    const double f = nd > t * nv ? 2.0 : (nv > t * nd ? 0.5 : 1.0);
    const double m = mu[img];
    mu_prev[img] = m;
    mu[img] = f * m;
    dscale[img] = 1.0 / f;
  }
}

__global__ void mu_fill_kernel(double *mu, double *mu_prev, double *dscale, int n, double mu0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    mu[i] = mu0;
    mu_prev[i] = mu0;
    dscale[i] = 1.0;
  }
}

cudaError_t launch_mu_update(const ImageDesc *desc_dev, int nimg, const double *apart, double *mu, double *mu_prev,
                             double *dscale, double t, cudaStream_t s) {
  mu_update_kernel<<<nimg, 128, 0, s>>>(desc_dev, apart, mu, mu_prev, dscale, t);
  return cudaGetLastError();
}

cudaError_t launch_mu_fill(double *mu, double *mu_prev, double *dscale, int nimg, double mu0, cudaStream_t s) {
  mu_fill_kernel<<<(nimg + 127) / 128, 128, 0, s>>>(mu, mu_prev, dscale, nimg, mu0);
  return cudaGetLastError();
}

cudaError_t launch_stats_reduce(const ImageDesc *desc_dev, int nimg, const double *partials, double *stats,
                                int iters, int it, int *err, cudaStream_t s) {
  stats_reduce_kernel<<<nimg, 128, 0, s>>>(desc_dev, partials, stats, iters, it, err);
  return cudaGetLastError();
}

}  // namespace dcv
