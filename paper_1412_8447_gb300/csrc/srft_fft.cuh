// Fast application of the structured sampling matrix of Section 5.2,
// Eq. (5.2): Y = sqrt(m / l) R F D A without forming the l x m matrix.  The
// pieces here are host-and-device functions so that the transform's index
// logic can be exercised by a host program as well as by the kernel in
// srft.cu.
//
// F is the orthonormal DCT-II along A's columns.  An unnormalised DCT-II of
// a real x of length m equals Re(e^{-i pi f / (2m)} V_f) where V is the
// length-m DFT of x reordered as v_p = x_{2p} (first half), v_{m-1-p} =
// x_{2p+1} (Makhoul, IEEE Trans. ASSP 28 (1980)).  Two real columns a, b
// share one complex transform of z = v(a) + i v(b): V(a)_f = (Z_f +
// conj Z_{m-f}) / 2 and V(b)_f = (Z_f - conj Z_{m-f}) / (2i).
//
// The DFT is an in-place mixed-radix decimation-in-frequency (Sande-Tukey)
// transform over m = r_0 r_1 ... r_{s-1} with radices 4, 2, 3, 5, 7.  Stage
// j works on blocks of length L_j = m / (r_0 ... r_{j-1}): for each block b
// and offset k < L_j / r_j it takes the r_j elements k + q L_j / r_j, forms
// their r_j-point DFT, multiplies output p by e^{-2 pi i p k / L_j} and
// writes it back at k + p L_j / r_j.  After the last stage Z_f sits at the
// digit-reversed position of f (fft_pos), so the l sampled frequencies are
// read from there and no reordering pass is needed.
#pragma once

#include <cmath>
#include <cstdint>
#include <initializer_list>

namespace curid {

constexpr int kFftMaxStages = 32;

// Radices of m in stage order; nst == -1 when m has a prime factor above 7.
struct FftPlan {
  int nst;
  int radix[kFftMaxStages];
};

inline FftPlan fft_plan(int64_t m) {
  FftPlan p{};
  p.nst = 0;
  for (int r : {4, 2, 3, 5, 7})
    while (m % r == 0 && p.nst < kFftMaxStages) {
      p.radix[p.nst++] = r;
      m /= r;
    }
  if (m != 1) p.nst = -1;
  return p;
}

// Where the in-place transform leaves Z_f: with f = p_0 + r_0 (p_1 + r_1
// (p_2 + ...)), position sum_j p_j m / (r_0 ... r_j).
__host__ __device__ inline int fft_pos(int f, const FftPlan& P, int m) {
  int pos = 0, rem = m;
  for (int j = 0; j < P.nst; ++j) {
    const int r = P.radix[j];
    rem /= r;
    pos += (f % r) * rem;
    f /= r;
  }
  return pos;
}

// Position of row t of the input after the even-odd reordering.
__host__ __device__ inline int fft_reorder(int t, int m) {
  return (t & 1) ? m - 1 - (t >> 1) : (t >> 1);
}

template <typename real>
struct cplx {
  real re, im;
};

template <typename real>
__host__ __device__ inline cplx<real> c_add(cplx<real> a, cplx<real> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename real>
__host__ __device__ inline cplx<real> c_sub(cplx<real> a, cplx<real> b) {
  return {a.re - b.re, a.im - b.im};
}
template <typename real>
__host__ __device__ inline cplx<real> c_mul(cplx<real> a, cplx<real> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename real>
__host__ __device__ inline cplx<real> c_scale(cplx<real> a, real s) {
  return {a.re * s, a.im * s};
}
// a - i b and a + i b
template <typename real>
__host__ __device__ inline cplx<real> c_sub_i(cplx<real> a, cplx<real> b) {
  return {a.re + b.im, a.im - b.re};
}
template <typename real>
__host__ __device__ inline cplx<real> c_add_i(cplx<real> a, cplx<real> b) {
  return {a.re - b.im, a.im + b.re};
}

// e^{-2 pi i k / L}, 0 <= k < L
template <typename real>
__host__ __device__ inline cplx<real> fft_twiddle(int k, int L) {
#ifdef __CUDA_ARCH__
  if constexpr (sizeof(real) == 4) {
    float s, c;
    // angle as a fraction of pi in (-1, 1]: k / L in [0, 1) folded to (-1/2, 1/2]
    const int kk = 2 * k > L ? k - L : k;
    sincospif(2.0f * (float)kk / (float)L, &s, &c);
    return {c, -s};
  } else {
    double s, c;
    const int kk = 2 * k > L ? k - L : k;
    sincospi(2.0 * (double)kk / (double)L, &s, &c);
    return {c, -s};
  }
#else
  const double a = 2.0 * 3.14159265358979323846 * (double)k / (double)L;
  return {(real)std::cos(a), (real)-std::sin(a)};
#endif
}

// r-point DFTs in registers, y_p = sum_q x_q e^{-2 pi i p q / r}.  Odd r use
// the pairs a_q = x_q + x_{r-q}, b_q = x_q - x_{r-q}: y_p = x_0 + sum_q a_q
// cos(2 pi p q / r) - i sum_q b_q sin(2 pi p q / r), y_{r-p} the same with +i.
template <typename real, int R>
struct Dft;

template <typename real>
struct Dft<real, 2> {
  __host__ __device__ static inline void run(cplx<real> (&x)[2]) {
    const cplx<real> a = x[0], b = x[1];
    x[0] = c_add(a, b);
    x[1] = c_sub(a, b);
  }
};

template <typename real>
struct Dft<real, 4> {
  __host__ __device__ static inline void run(cplx<real> (&x)[4]) {
    const cplx<real> s02 = c_add(x[0], x[2]), d02 = c_sub(x[0], x[2]);
    const cplx<real> s13 = c_add(x[1], x[3]), d13 = c_sub(x[1], x[3]);
    x[0] = c_add(s02, s13);
    x[2] = c_sub(s02, s13);
    x[1] = c_sub_i(d02, d13);
    x[3] = c_add_i(d02, d13);
  }
};

template <typename real>
struct Dft<real, 3> {
  __host__ __device__ static inline void run(cplx<real> (&x)[3]) {
    const real c1 = (real)-0.5, s1 = (real)0.86602540378443864676;
    const cplx<real> a = c_add(x[1], x[2]), b = c_sub(x[1], x[2]);
    const cplx<real> A = c_add(x[0], c_scale(a, c1)), B = c_scale(b, s1);
    x[0] = c_add(x[0], a);
    x[1] = c_sub_i(A, B);
    x[2] = c_add_i(A, B);
  }
};

template <typename real>
struct Dft<real, 5> {
  __host__ __device__ static inline void run(cplx<real> (&x)[5]) {
    const real c1 = (real)0.30901699437494742410, s1 = (real)0.95105651629515357212;
    const real c2 = (real)-0.80901699437494742410, s2 = (real)0.58778525229247312917;
    const cplx<real> a1 = c_add(x[1], x[4]), b1 = c_sub(x[1], x[4]);
    const cplx<real> a2 = c_add(x[2], x[3]), b2 = c_sub(x[2], x[3]);
    // p = 1: angles 1, 2; p = 2: angles 2, 4 (cos 4 = cos 1, sin 4 = -sin 1)
    const cplx<real> A1 = c_add(x[0], c_add(c_scale(a1, c1), c_scale(a2, c2)));
    const cplx<real> B1 = c_add(c_scale(b1, s1), c_scale(b2, s2));
    const cplx<real> A2 = c_add(x[0], c_add(c_scale(a1, c2), c_scale(a2, c1)));
    const cplx<real> B2 = c_sub(c_scale(b1, s2), c_scale(b2, s1));
    x[0] = c_add(x[0], c_add(a1, a2));
    x[1] = c_sub_i(A1, B1);
    x[4] = c_add_i(A1, B1);
    x[2] = c_sub_i(A2, B2);
    x[3] = c_add_i(A2, B2);
  }
};

template <typename real>
struct Dft<real, 7> {
  __host__ __device__ static inline void run(cplx<real> (&x)[7]) {
    const real c1 = (real)0.62348980185873353053, s1 = (real)0.78183148246802980871;
    const real c2 = (real)-0.22252093395631440429, s2 = (real)0.97492791218182360702;
    const real c3 = (real)-0.90096886790241912624, s3 = (real)0.43388373911755812048;
    const cplx<real> a1 = c_add(x[1], x[6]), b1 = c_sub(x[1], x[6]);
    const cplx<real> a2 = c_add(x[2], x[5]), b2 = c_sub(x[2], x[5]);
    const cplx<real> a3 = c_add(x[3], x[4]), b3 = c_sub(x[3], x[4]);
    // angle p q mod 7: p = 1 -> 1, 2, 3; p = 2 -> 2, 4, 6; p = 3 -> 3, 6, 2
    // (cos(7 - j) = cos j, sin(7 - j) = -sin j)
    const cplx<real> A1 =
        c_add(x[0], c_add(c_scale(a1, c1), c_add(c_scale(a2, c2), c_scale(a3, c3))));
    const cplx<real> B1 = c_add(c_scale(b1, s1), c_add(c_scale(b2, s2), c_scale(b3, s3)));
    const cplx<real> A2 =
        c_add(x[0], c_add(c_scale(a1, c2), c_add(c_scale(a2, c3), c_scale(a3, c1))));
    const cplx<real> B2 = c_sub(c_scale(b1, s2), c_add(c_scale(b2, s3), c_scale(b3, s1)));
    const cplx<real> A3 =
        c_add(x[0], c_add(c_scale(a1, c3), c_add(c_scale(a2, c1), c_scale(a3, c2))));
    const cplx<real> B3 = c_add(c_sub(c_scale(b1, s3), c_scale(b2, s1)), c_scale(b3, s2));
    x[0] = c_add(x[0], c_add(a1, c_add(a2, a3)));
    x[1] = c_sub_i(A1, B1);
    x[6] = c_add_i(A1, B1);
    x[2] = c_sub_i(A2, B2);
    x[5] = c_add_i(A2, B2);
    x[3] = c_sub_i(A3, B3);
    x[4] = c_add_i(A3, B3);
  }
};

// One stage of radix R over NS sequences of length m stored one after the
// other in z, block length L; butterflies u = first, first + step, ...
template <typename real, int R, int NS>
__host__ __device__ inline void fft_stage(cplx<real>* z, int m, int L, int first, int step) {
  const int span = L / R;
  const int nb = m / R;
  for (int u = first; u < nb; u += step) {
    const int b = u / span, k = u - b * span;
    const int base = b * L + k;
    cplx<real> w[R];
    w[0] = {(real)1, (real)0};
    if (R > 1) w[1] = fft_twiddle<real>(k, L);
#pragma unroll
    for (int p = 2; p < R; ++p) w[p] = c_mul(w[p - 1], w[1]);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      cplx<real>* zs = z + (int64_t)s * m + base;
      cplx<real> x[R];
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = zs[q * span];
      Dft<real, R>::run(x);
      zs[0] = x[0];
#pragma unroll
      for (int p = 1; p < R; ++p) zs[p * span] = c_mul(x[p], w[p]);
    }
  }
}

// Row f of the sampled transform for the two real columns held in z (one
// sequence): writes the unscaled DCT-II values of both.  f is reduced with
// the periodic extension of F: rows f and 4m - f agree, row 2m - f is minus
// row f, row m is zero.  Returns the sign to apply.
template <typename real>
__host__ __device__ inline real fft_dct_pair(const cplx<real>* z, const FftPlan& P, int m,
                                            int64_t f_in, real* x1, real* x2) {
  const int64_t four_m = 4LL * m;
  int64_t f = ((f_in % four_m) + four_m) % four_m;
  real sg = (real)1;
  if (f > 2LL * m) f = four_m - f;
  if (f > m) {
    f = 2LL * m - f;
    sg = (real)-1;
  }
  // f in [0, m]; V is periodic with period m
  const int fm = (int)(f % m);
  const int fc = fm == 0 ? 0 : m - fm;
  const cplx<real> Zf = z[fft_pos(fm, P, m)];
  const cplx<real> Zc = z[fft_pos(fc, P, m)];
  // conj(Zc): (Zc.re, -Zc.im)
  const cplx<real> V1 = {(real)0.5 * (Zf.re + Zc.re), (real)0.5 * (Zf.im - Zc.im)};
  // (Zf - conj Zc) / (2i) = (d.im / 2, -d.re / 2)
  const cplx<real> d = {Zf.re - Zc.re, Zf.im + Zc.im};
  const cplx<real> V2 = {(real)0.5 * d.im, (real)-0.5 * d.re};
  real c, s;
#ifdef __CUDA_ARCH__
  if constexpr (sizeof(real) == 4) {
    sincospif((float)f / (float)(2 * m), &s, &c);
  } else {
    sincospi((double)f / (double)(2 * m), &s, &c);
  }
#else
  const double a = 3.14159265358979323846 * (double)f / (2.0 * m);
  c = (real)std::cos(a);
  s = (real)std::sin(a);
#endif
  *x1 = c * V1.re + s * V1.im;
  *x2 = c * V2.re + s * V2.im;
  return sg;
}

}  // namespace curid
