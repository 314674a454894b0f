// FFTs of the row and column passes: register-resident transforms (fft_p2,
// fft_mixed, fft_v16, further below) for lengths 2^k, 3 * 2^k and 5 * 2^k,
// and a shared-memory mixed-radix Stockham transform for any other
// 2^a 3^b 5^c length (first part of this file).
//
// The 2-D DFT that diagonalises T~^T T~ + mu D^T D (Sec. II-B, the paragraph
// after the over-relaxed z-update) is computed as 1-D transforms along rows
// and along columns.  Each CTA holds a batch of S signals of length L in
// shared memory, laid out [position][signal] with an odd leading dimension
// `ld` (signal index fastest, so consecutive threads touch consecutive
// addresses and an odd stride avoids bank conflicts on the transposing
// writes).  The transform is an in-place Stockham auto-sort sequence of
// radix-R passes (R in {2,3,4,5,8,16}, chosen per length on the host): in
// pass p with span Ns (the product of the radices already applied), the
// butterfly j reads elements j + r L/R, multiplies element r by
// w^(r (j mod Ns)) with w = exp(sign 2 pi i / (Ns R)), applies an R-point
// DFT in registers and writes element r to (j - j mod Ns) R + j mod Ns +
// r Ns.  After the last pass the output is in natural order (the Stockham
// formulation of Govindaraju et al., SC'08, written for [position][signal]
// storage).  Each thread
// keeps at most 32 complex values in registers per pass, so a CTA of NT
// threads can hold S * L <= 30 NT elements.
//
// Twiddles come from a table tw[m] = exp(-2 pi i m / L) computed on the host
// in double precision (cos/sin of the exact rational angle) and rounded once
// to the element type; the inverse uses the conjugate.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dcv {

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T> using cx = typename vec2<T>::type;

template <typename T> __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename T> __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by sign * i
template <typename T, int SIGN> __device__ __forceinline__ cx<T> mul_si(cx<T> a) {
  return SIGN > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// R-point DFTs in registers: X[q] = sum_r v[r] exp(SIGN 2 pi i r q / R).
// Constants are the exact values of cos/sin at multiples of 2 pi / R.

template <typename T, int R, int SIGN> struct Dft;

template <typename T, int SIGN> struct Dft<T, 2, SIGN> {
  static __device__ __forceinline__ void run(cx<T> *v) {
    cx<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  }
};

template <typename T, int SIGN> struct Dft<T, 3, SIGN> {
  static __device__ __forceinline__ void run(cx<T> *v) {
    const T c = T(-0.5), s = T(0.86602540378443864676);  // cos, |sin| of 2 pi / 3
    cx<T> t1 = cadd<T>(v[1], v[2]), t2 = csub<T>(v[1], v[2]);
    cx<T> m = mk<T>(v[0].x + c * t1.x, v[0].y + c * t1.y);
    cx<T> r = mul_si<T, SIGN>(cscale<T>(t2, s));
    v[0] = cadd<T>(v[0], t1);
    v[1] = cadd<T>(m, r);
    v[2] = csub<T>(m, r);
  }
};

template <typename T, int SIGN> struct Dft<T, 4, SIGN> {
  static __device__ __forceinline__ void run(cx<T> *v) {
    cx<T> a = cadd<T>(v[0], v[2]), b = csub<T>(v[0], v[2]);
    cx<T> c = cadd<T>(v[1], v[3]), d = mul_si<T, SIGN>(csub<T>(v[1], v[3]));
    v[0] = cadd<T>(a, c);
    v[2] = csub<T>(a, c);
    v[1] = cadd<T>(b, d);
    v[3] = csub<T>(b, d);
  }
};

template <typename T, int SIGN> struct Dft<T, 5, SIGN> {
  static __device__ __forceinline__ void run(cx<T> *v) {
    const T c1 = T(0.30901699437494742410), s1 = T(0.95105651629515357212);   // 2 pi / 5
    const T c2 = T(-0.80901699437494742410), s2 = T(0.58778525229247312917);  // 4 pi / 5
    cx<T> a1 = cadd<T>(v[1], v[4]), b1 = csub<T>(v[1], v[4]);
    cx<T> a2 = cadd<T>(v[2], v[3]), b2 = csub<T>(v[2], v[3]);
    cx<T> m1 = mk<T>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    cx<T> m2 = mk<T>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    cx<T> r1 = mul_si<T, SIGN>(mk<T>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
    cx<T> r2 = mul_si<T, SIGN>(mk<T>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
    v[0] = mk<T>(v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y);
    v[1] = cadd<T>(m1, r1);
    v[4] = csub<T>(m1, r1);
    v[2] = cadd<T>(m2, r2);
    v[3] = csub<T>(m2, r2);
  }
};

// 8 = 2 x 4 (even/odd split), 16 = 2 x 8.
template <typename T, int SIGN> struct Dft<T, 8, SIGN> {
  static __device__ __forceinline__ void run(cx<T> *v) {
    const T h = T(0.70710678118654752440);
    cx<T> e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, 4, SIGN>::run(e);
    Dft<T, 4, SIGN>::run(o);
    // w8^q, q = 0..3, w8 = exp(SIGN i pi / 4)
    cx<T> t1 = cmul<T>(o[1], mk<T>(h, SIGN * h));
    cx<T> t2 = mul_si<T, SIGN>(o[2]);
    cx<T> t3 = cmul<T>(o[3], mk<T>(-h, SIGN * h));
    v[0] = cadd<T>(e[0], o[0]);
    v[4] = csub<T>(e[0], o[0]);
    v[1] = cadd<T>(e[1], t1);
    v[5] = csub<T>(e[1], t1);
    v[2] = cadd<T>(e[2], t2);
    v[6] = csub<T>(e[2], t2);
    v[3] = cadd<T>(e[3], t3);
    v[7] = csub<T>(e[3], t3);
  }
};

template <typename T, int SIGN> struct Dft<T, 16, SIGN> {
  static __device__ __forceinline__ void run(cx<T> *v) {
    // cos, sin of q pi / 8 for q = 0..7
    const T C[8] = {T(1.0), T(0.92387953251128675613), T(0.70710678118654752440), T(0.38268343236508977173),
                    T(0.0), T(-0.38268343236508977173), T(-0.70710678118654752440), T(-0.92387953251128675613)};
    const T S[8] = {T(0.0), T(0.38268343236508977173), T(0.70710678118654752440), T(0.92387953251128675613),
                    T(1.0), T(0.92387953251128675613), T(0.70710678118654752440), T(0.38268343236508977173)};
    cx<T> e[8], o[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      e[r] = v[2 * r];
      o[r] = v[2 * r + 1];
    }
    Dft<T, 8, SIGN>::run(e);
    Dft<T, 8, SIGN>::run(o);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      cx<T> t = (q == 0) ? o[0] : cmul<T>(o[q], mk<T>(C[q], SIGN * S[q]));
      v[q] = cadd<T>(e[q], t);
      v[q + 8] = csub<T>(e[q], t);
    }
  }
};

template <typename T, int SIGN> struct Dft<T, 1, SIGN> {
  static __device__ __forceinline__ void run(cx<T> *) {}
};

// 32 = 2 x 16.
template <typename T, int SIGN> struct Dft<T, 32, SIGN> {
  static __device__ __forceinline__ void run(cx<T> *v) {
    // cos, sin of q pi / 16 for q = 0..15
    const T C[16] = {T(1.0), T(0.98078528040323044913), T(0.92387953251128675613), T(0.83146961230254523708),
                     T(0.70710678118654752440), T(0.55557023301960222474), T(0.38268343236508977173),
                     T(0.19509032201612826785), T(0.0), T(-0.19509032201612826785), T(-0.38268343236508977173),
                     T(-0.55557023301960222474), T(-0.70710678118654752440), T(-0.83146961230254523708),
                     T(-0.92387953251128675613), T(-0.98078528040323044913)};
    const T S[16] = {T(0.0), T(0.19509032201612826785), T(0.38268343236508977173), T(0.55557023301960222474),
                     T(0.70710678118654752440), T(0.83146961230254523708), T(0.92387953251128675613),
                     T(0.98078528040323044913), T(1.0), T(0.98078528040323044913), T(0.92387953251128675613),
                     T(0.83146961230254523708), T(0.70710678118654752440), T(0.55557023301960222474),
                     T(0.38268343236508977173), T(0.19509032201612826785)};
    cx<T> e[16], o[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      e[r] = v[2 * r];
      o[r] = v[2 * r + 1];
    }
    Dft<T, 16, SIGN>::run(e);
    Dft<T, 16, SIGN>::run(o);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      cx<T> t = (q == 0) ? o[0] : (q == 8 ? mul_si<T, SIGN>(o[8]) : cmul<T>(o[q], mk<T>(C[q], SIGN * S[q])));
      v[q] = cadd<T>(e[q], t);
      v[q + 16] = csub<T>(e[q], t);
    }
  }
};

// ---------------------------------------------------------------------------
// Register-resident transform of length L = 32 TT by a group of TT threads
// (TT in {1, 2, 4, 8, 16, 32}; a group never spans two warps).  Index split
// n = t + TT m (t < TT, m < 32), k = k1 + 32 k2 (k1 < 32, k2 < TT):
//   X[k1 + 32 k2] = sum_t w_TT^(t k2) [ w_L^(t k1) sum_m x[t + TT m] w_32^(m k1) ],
// the two-factor Cooley-Tukey split.  Thread q of the group enters with
// v[m] = x[q + TT m] and leaves with v[j TT + k2] = X[q + TT j + 32 k2]
// (j < 32/TT), i.e. v[r] holds index q + TT * p2_slot(r).  Step 1 is a 32-point
// DFT in registers, then one twiddle multiply from a table laid out
// [k1][t] (coalesced), one transpose through the group's shared tile, and
// TT-point DFTs in registers.  The tile is padded (row stride TT+1, group
// stride p2_group_stride) so the transposing accesses are free of bank
// conflicts.
template <int TT> __host__ __device__ constexpr int p2_group_stride() {
  return 32 * (TT + 1) + (TT < 16 ? TT : 0);
}
__host__ __device__ constexpr int p2_group_stride_h(int tt) { return 32 * (tt + 1) + (tt < 16 ? tt : 0); }

// Position index m of register r after the transform (see above).
template <int TT> __device__ __forceinline__ constexpr int p2_slot(int r) {
  return (r / TT) + (32 / TT) * (r % TT);
}

template <typename T, int TT, int SIGN>
__device__ __forceinline__ void fft_p2(cx<T> (&v)[32], cx<T> *tile, int q, unsigned gmask,
                                       const cx<T> *__restrict__ tw2) {
  Dft<T, 32, SIGN>::run(v);
  if constexpr (TT > 1) {
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) {
      cx<T> w = __ldg(&tw2[k1 * TT + q]);
      if (SIGN > 0) w.y = -w.y;
      v[k1] = cmul<T>(v[k1], w);
    }
    constexpr int LD = TT + 1;
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) tile[k1 * LD + q] = v[k1];
    __syncwarp(gmask);
#pragma unroll
    for (int j = 0; j < 32 / TT; ++j) {
#pragma unroll
      for (int t = 0; t < TT; ++t) v[j * TT + t] = tile[(q + TT * j) * LD + t];
      Dft<T, TT, SIGN>::run(&v[j * TT]);
    }
    __syncwarp(gmask);
  }
}

// ---------------------------------------------------------------------------
// Mixed transform of length L = R * L2, L2 = 32 TT, R in {1, 3, 5}, by R
// groups of TT threads (decimation in time: x[R n2 + r] -> F_r).  Group gr
// enters with v[m] = x[R (q + TT m) + gr] and leaves with
// v[j] = X[q + TT p2_slot(j) + L2 gr].  Steps: the L2-point transform of its
// sub-sequence (fft_p2), the twiddle w^(gr k2) (table tw3 laid out [r][k2],
// w = exp(-2 pi i / L), conjugated for the inverse) into the exchange buffer
// E (L complex, this transform's), and the R-point combine
// X[k2 + L2 s] = sum_r E[r][k2] exp(SIGN 2 pi i r s / R) for s = gr.
// Contains __syncthreads when R > 1: every thread of the CTA must call it
// (threads of inactive groups with active = false).  E may share storage
// with the R groups' transpose tiles (a barrier separates their uses).
template <typename T, int R, int SIGN> __device__ __forceinline__ cx<T> root_r(int j) {
  // exp(SIGN 2 pi i j / R) for R = 3, 5 (exact constants)
  if constexpr (R == 3) {
    const T s3 = T(0.86602540378443864676);
    return j == 0 ? mk<T>(T(1), T(0)) : (j == 1 ? mk<T>(T(-0.5), SIGN * s3) : mk<T>(T(-0.5), -SIGN * s3));
  } else {
    const T c1 = T(0.30901699437494742410), s1 = T(0.95105651629515357212);
    const T c2 = T(-0.80901699437494742410), s2 = T(0.58778525229247312917);
    switch (j) {
      case 0: return mk<T>(T(1), T(0));
      case 1: return mk<T>(c1, SIGN * s1);
      case 2: return mk<T>(c2, SIGN * s2);
      case 3: return mk<T>(c2, -SIGN * s2);
      default: return mk<T>(c1, -SIGN * s1);
    }
  }
}

template <typename T, int TT, int R, int SIGN>
__device__ __forceinline__ void fft_mixed(cx<T> (&v)[32], bool active, cx<T> *tile, int q, unsigned gmask, int gr,
                                          const cx<T> *__restrict__ tw2, const cx<T> *__restrict__ tw3, cx<T> *E) {
  constexpr int L2 = 32 * TT;
  if (active) fft_p2<T, TT, SIGN>(v, tile, q, gmask, tw2);
  if constexpr (R > 1) {
    __syncthreads();  // E may overlay the transpose tiles of the other groups
    if (active) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int k2 = q + TT * p2_slot<TT>(j);
        cx<T> w = __ldg(&tw3[gr * L2 + k2]);
        if (SIGN > 0) w.y = -w.y;
        E[gr * L2 + k2] = cmul<T>(v[j], w);
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int k2 = q + TT * p2_slot<TT>(j);
        cx<T> acc = E[k2];
#pragma unroll
        for (int r = 1; r < R; ++r) acc = cadd<T>(acc, cmul<T>(E[r * L2 + k2], root_r<T, R, SIGN>((r * gr) % R)));
        v[j] = acc;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Register-resident transform of length L = 16 TT by TT threads holding 16
// complex values each (TT in {1, 2, 4, 8, 16, 32, 64}): twice the threads of
// fft_p2 for the same length, so twice the resident warps for a pass whose
// parallelism is its row or column count.  Index split n = q + TT m
// (q < TT, m < 16), k = k1 + 16 k2: a 16-point DFT in registers, the twiddle
// w_L^(q k1) from a [k1][q] table, then the TT-point DFTs over q for every
// k1: for TT <= 16 one transpose through the group's tile and TT-point DFTs
// in registers; for TT = A B (A = 4 or 8, B = TT / A) two transposes with a
// B-point stage, the twiddle w_TT^(a c) ([a][c] table) and an A-point stage
// (k2 = c + B d; the TT-point index splits as a + A b).  Thread q enters with v[m] = x[q + TT m] and
// leaves with v[r] = X[v16_pos<TT>(q, r)].  Groups of 64 threads span two
// warps and synchronise with the named barrier `bar` (1..15).
template <int TT> __device__ __forceinline__ void group_bar(unsigned gmask, int bar) {
  if constexpr (TT <= 32)
    __syncwarp(gmask);
  else
    asm volatile("bar.sync %0, %1;\n" ::"r"(bar), "n"(TT) : "memory");
}

template <int TT> __host__ __device__ constexpr int v16_A() { return TT == 64 ? 8 : 4; }

// Output position of register r of thread q (see fft_v16).
template <int TT> __device__ __forceinline__ int v16_pos(int q, int r) {
  if constexpr (TT <= 16) {
    return q + TT * (r / TT + (16 / TT) * (r % TT));
  } else {
    constexpr int A = v16_A<TT>(), B = TT / A;
    return q % 16 + 16 * ((q / 16) * (16 / A) + r / A + B * (r % A));
  }
}

// Tiles of the two-transpose path (complex elements), laid out so that the
// 32 lanes of every transposing access spread over all 16 bank pairs: the
// first [k1][q] with row stride LD1 (TT = 32: 36, 64: 72), the second
// [c][a][k1] with strides L16 for a (32: 24, 64: 20) and A L16 for c.
__host__ __device__ constexpr int v16_ld1(int tt) { return tt == 64 ? 72 : 36; }
__host__ __device__ constexpr int v16_l16(int tt) { return tt == 64 ? 20 : 24; }

// Shared tile of one group (complex elements).
__host__ __device__ constexpr int v16_group_stride_h(int tt) {
  return tt <= 16 ? 16 * (tt + 1) + (tt < 16 ? tt : 0) : tt * v16_l16(tt);  // B * (A * L16)
}
template <int TT> __host__ __device__ constexpr int v16_group_stride() { return v16_group_stride_h(TT); }

template <typename T, int TT, int SIGN>
__device__ __forceinline__ void fft_v16(cx<T> (&v)[16], cx<T> *tile, int q, unsigned gmask, int bar,
                                        const cx<T> *__restrict__ tw16, const cx<T> *__restrict__ twab) {
  Dft<T, 16, SIGN>::run(v);
  if constexpr (TT > 1) {
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
      cx<T> w = __ldg(&tw16[k1 * TT + q]);
      if (SIGN > 0) w.y = -w.y;
      v[k1] = cmul<T>(v[k1], w);
    }
    if constexpr (TT <= 16) {
      constexpr int LD = TT + 1;
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) tile[k1 * LD + q] = v[k1];
      group_bar<TT>(gmask, bar);
#pragma unroll
      for (int j = 0; j < 16 / TT; ++j) {
#pragma unroll
        for (int t = 0; t < TT; ++t) v[j * TT + t] = tile[(q + TT * j) * LD + t];
        Dft<T, TT, SIGN>::run(&v[j * TT]);
      }
      group_bar<TT>(gmask, bar);
    } else {
      // stage 2 takes (k1, a) = (b + B i, q mod A), stage 3 takes (k1, c) =
      // (q mod 16, (q / 16) (16 / A) + i)
      constexpr int A = v16_A<TT>(), B = TT / A, LD1 = v16_ld1(TT), L16 = v16_l16(TT), S2 = A * L16;
      const int a = q % A, b = q / A;
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) tile[k1 * LD1 + q] = v[k1];
      group_bar<TT>(gmask, bar);
#pragma unroll
      for (int i = 0; i < 16 / B; ++i)
#pragma unroll
        for (int b2 = 0; b2 < B; ++b2) v[i * B + b2] = tile[(b + B * i) * LD1 + a + A * b2];
      group_bar<TT>(gmask, bar);
#pragma unroll
      for (int i = 0; i < 16 / B; ++i) Dft<T, B, SIGN>::run(&v[i * B]);
#pragma unroll
      for (int c = 1; c < B; ++c) {
        cx<T> w = __ldg(&twab[a * B + c]);
        if (SIGN > 0) w.y = -w.y;
#pragma unroll
        for (int i = 0; i < 16 / B; ++i) v[i * B + c] = cmul<T>(v[i * B + c], w);
      }
#pragma unroll
      for (int i = 0; i < 16 / B; ++i)
#pragma unroll
        for (int c = 0; c < B; ++c) tile[c * S2 + a * L16 + b + B * i] = v[i * B + c];
      group_bar<TT>(gmask, bar);
      const int k1 = q % 16, f = q / 16;
#pragma unroll
      for (int i = 0; i < 16 / A; ++i)
#pragma unroll
        for (int a2 = 0; a2 < A; ++a2) v[i * A + a2] = tile[(f * (16 / A) + i) * S2 + a2 * L16 + k1];
      group_bar<TT>(gmask, bar);
#pragma unroll
      for (int i = 0; i < 16 / A; ++i) Dft<T, A, SIGN>::run(&v[i * A]);
    }
  }
}

// ---------------------------------------------------------------------------
// One radix-R Stockham pass over S signals of length L held in buf.  The
// host plans S * L <= 30 NT so that every butterfly has a register slot.
template <typename T, int NT, int R, int SIGN>
__device__ __forceinline__ void stockham_pass(cx<T> *buf, int L, int S, int ld, int Ns,
                                              const cx<T> *__restrict__ tw) {
  constexpr int CM = 32 / R;
  const int LR = L / R;
  const int nbf = S * LR;
  const int tstride = L / (Ns * R);
  cx<T> v[CM][R];
#pragma unroll
  for (int c = 0; c < CM; ++c) {
    const int b = threadIdx.x + c * NT;
    if (b < nbf) {
      const int s = b % S, j = b / S, k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = buf[(j + r * LR) * ld + s];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cx<T> w = __ldg(&tw[k * r * tstride]);
          if (SIGN > 0) w.y = -w.y;
          v[c][r] = cmul<T>(v[c][r], w);
        }
      }
      Dft<T, R, SIGN>::run(v[c]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CM; ++c) {
    const int b = threadIdx.x + c * NT;
    if (b < nbf) {
      const int s = b % S, j = b / S, k = j % Ns;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[(base + r * Ns) * ld + s] = v[c][r];
    }
  }
  __syncthreads();
}

// Radix schedule of one length L = 16^n16 * r * 5^n5 * 3^n3 with r in
// {1, 2, 4, 8}: the passes run in that fixed order.  (A fixed sequence of
// pass loops, instead of one loop over a runtime radix switch, lets the
// register allocator treat each pass on its own.)
struct FftSched {
  int8_t n16, r, n5, n3;
};

// Full transform.  buf must be complete (a __syncthreads after it was
// written) on entry; it is complete on return.
template <typename T, int NT, int SIGN>
__device__ __forceinline__ void fft_smem(cx<T> *buf, int L, int S, int ld, FftSched sc,
                                         const cx<T> *__restrict__ tw) {
  int Ns = 1;
  for (int p = 0; p < sc.n16; ++p) {
    stockham_pass<T, NT, 16, SIGN>(buf, L, S, ld, Ns, tw);
    Ns *= 16;
  }
  if (sc.r == 8) {
    stockham_pass<T, NT, 8, SIGN>(buf, L, S, ld, Ns, tw);
    Ns *= 8;
  } else if (sc.r == 4) {
    stockham_pass<T, NT, 4, SIGN>(buf, L, S, ld, Ns, tw);
    Ns *= 4;
  } else if (sc.r == 2) {
    stockham_pass<T, NT, 2, SIGN>(buf, L, S, ld, Ns, tw);
    Ns *= 2;
  }
  for (int p = 0; p < sc.n5; ++p) {
    stockham_pass<T, NT, 5, SIGN>(buf, L, S, ld, Ns, tw);
    Ns *= 5;
  }
  for (int p = 0; p < sc.n3; ++p) {
    stockham_pass<T, NT, 3, SIGN>(buf, L, S, ld, Ns, tw);
    Ns *= 3;
  }
}

}  // namespace dcv
