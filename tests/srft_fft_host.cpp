// Host build of the fast structured-sample transform (srft_fft.cuh) for the
// CPU tests: the same stage, position and DCT-extraction functions the
// kernel runs, driven serially.  Reads from stdin "m ncols l prec", then A
// (m x ncols, row major), the m signs and the l rows; prints Y (l x ncols).
// prec 0: double, 1: float.  ncols is 2 (one complex sequence) or 4 (two).
#define __host__
#define __device__
#include "../paper_1412_8447_gb300/csrc/srft_fft.cuh"

#include <cstdio>
#include <vector>

using namespace curid;

template <typename real, int NS>
static int run(int m, int l, const std::vector<double>& A, const std::vector<int>& sg,
               const std::vector<long long>& rows) {
  const FftPlan P = fft_plan(m);
  if (P.nst < 0) {
    std::printf("unsupported\n");
    return 0;
  }
  const int nc = 2 * NS;
  std::vector<cplx<real>> z((size_t)NS * m);
  for (int t = 0; t < m; ++t) {
    const int p = fft_reorder(t, m);
    const real d = sg[t] < 0 ? (real)-1 : (real)1;
    for (int s = 0; s < NS; ++s)
      z[(size_t)s * m + p] = {(real)A[(size_t)t * nc + 2 * s] * d,
                              (real)A[(size_t)t * nc + 2 * s + 1] * d};
  }
  int L = m;
  for (int j = 0; j < P.nst; ++j) {
    const int r = P.radix[j];
    // three interleaved "threads", as a block of threads would split the butterflies
    for (int th = 0; th < 3; ++th) {
      switch (r) {
        case 4: fft_stage<real, 4, NS>(z.data(), m, L, th, 3); break;
        case 2: fft_stage<real, 2, NS>(z.data(), m, L, th, 3); break;
        case 3: fft_stage<real, 3, NS>(z.data(), m, L, th, 3); break;
        case 5: fft_stage<real, 5, NS>(z.data(), m, L, th, 3); break;
        default: fft_stage<real, 7, NS>(z.data(), m, L, th, 3); break;
      }
    }
    L /= r;
  }
  const long long four_m = 4LL * m;
  for (int i = 0; i < l; ++i) {
    const long long f0 = ((rows[i] % four_m) + four_m) % four_m;
    const real sc = (real)std::sqrt((f0 == 0 ? 1.0 : 2.0) / l);
    for (int s = 0; s < NS; ++s) {
      real x1, x2;
      const real g = fft_dct_pair<real>(z.data() + (size_t)s * m, P, m, rows[i], &x1, &x2);
      std::printf("%.17g %.17g ", (double)(g * sc * x1), (double)(g * sc * x2));
    }
    std::printf("\n");
  }
  return 0;
}

int main() {
  int m, nc, l, prec;
  if (std::scanf("%d %d %d %d", &m, &nc, &l, &prec) != 4) return 1;
  std::vector<double> A((size_t)m * nc);
  for (auto& v : A)
    if (std::scanf("%lf", &v) != 1) return 1;
  std::vector<int> sg(m);
  for (auto& v : sg)
    if (std::scanf("%d", &v) != 1) return 1;
  std::vector<long long> rows(l);
  for (auto& v : rows)
    if (std::scanf("%lld", &v) != 1) return 1;
  if (nc == 2) return prec ? run<float, 1>(m, l, A, sg, rows) : run<double, 1>(m, l, A, sg, rows);
  return prec ? run<float, 2>(m, l, A, sg, rows) : run<double, 2>(m, l, A, sg, rows);
}
