// Gaussian test matrix Omega (Algorithm 4, line 1; Section 5.1: i.i.d.
// standard Gaussian entries).
// Counter-based generator Philox4x32-10 as published by Salmon, Moraes,
// Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC'11):
// a 4 x 32-bit counter and 2 x 32-bit key, 10 rounds, each round two
// 32x32->64 multiplications by M0 = 0xD2511F53 and M1 = 0xCD9E8D57, the key
// bumped by the Weyl constants W0 = 0x9E3779B9, W1 = 0xBB67AE85 between
// rounds.  Words are mapped to uniforms in (0, 1] on a 2^-24 grid and paired
// by the Box-Muller transform.  Element e of the row-major matrix uses
// counter (e / 4, 0, 0, 0) and word e % 4: words (0, 1) give the cosine and
// sine branch of one pair, words (2, 3) of the next.  Element e = r*cols + c
// is stored at out[r*ld + c].
#include "kernels.cuh"

namespace curid {

namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 key) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ key.x, lo1, hi0 ^ c.w ^ key.y, lo0);
    key.x += 0x9E3779B9u;
    key.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ double u01(unsigned w) {
  return (double)((w >> 8) + 1u) * (1.0 / 16777216.0);
}

template <typename real>
__global__ void gaussian_kernel(int64_t total, int64_t cols, int64_t ld, uint2 key,
                                real* __restrict__ out) {
  const int64_t groups = (total + 3) / 4;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
       g += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((unsigned)g, (unsigned)(g >> 32), 0u, 0u), key);
    real z[4];
    if (sizeof(real) == 8) {
      const double r0 = sqrt(-2.0 * log(u01(w.x))), t0 = 6.283185307179586 * u01(w.y);
      const double r1 = sqrt(-2.0 * log(u01(w.z))), t1 = 6.283185307179586 * u01(w.w);
      z[0] = (real)(r0 * cos(t0));
      z[1] = (real)(r0 * sin(t0));
      z[2] = (real)(r1 * cos(t1));
      z[3] = (real)(r1 * sin(t1));
    } else {
      const float r0 = sqrtf(-2.0f * logf((float)u01(w.x))), t0 = 6.2831855f * (float)u01(w.y);
      const float r1 = sqrtf(-2.0f * logf((float)u01(w.z))), t1 = 6.2831855f * (float)u01(w.w);
      z[0] = (real)(r0 * cosf(t0));
      z[1] = (real)(r0 * sinf(t0));
      z[2] = (real)(r1 * cosf(t1));
      z[3] = (real)(r1 * sinf(t1));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t e = 4 * g + q;
      if (e < total) out[(e / cols) * ld + e % cols] = z[q];
    }
  }
}

// Random choices of the structured sampling matrix (Section 5.2, Eq. (5.2)):
// the m signs of D and the l rows R keeps, drawn without replacement.
// Sign t: top bit of word t % 4 of Philox4x32-10 at counter (t / 4, 0, 1, 0)
// (third counter word 1: a stream apart from the Gaussian generator's).
// Rows: rows[i] = pi(i) for a pseudo-random permutation pi of [0, m): a
// four-round balanced Feistel network on 2h-bit values (2^(2h) >= m) whose
// round function is Philox at counter (half-word, round, 2, 0), restricted to
// [0, m) by cycle walking (Black and Rogaway, "Ciphers with arbitrary finite
// domains", CT-RSA 2002): apply the network until the value falls below m.
// Distinct i give distinct rows because the restriction is itself a
// permutation.
__device__ __forceinline__ unsigned feistel(unsigned x, int h, uint2 key) {
  const unsigned mask = (1u << h) - 1u;
  unsigned L = x >> h, R = x & mask;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const unsigned F = philox4x32_10(make_uint4(R, (unsigned)r, 2u, 0u), key).x & mask;
    const unsigned nl = R;
    R = L ^ F;
    L = nl;
  }
  return (L << h) | R;
}

__global__ void srft_draw_kernel(int64_t m, int64_t l, int h, uint2 key, int32_t* __restrict__ rows,
                                 int8_t* __restrict__ signs) {
  const int64_t span = 1LL << (2 * h);  // the network's domain, < 4m
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m || e < l;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < m) {
      const uint4 w = philox4x32_10(
          make_uint4((unsigned)(e >> 2), (unsigned)(e >> 34), 1u, 0u), key);
      const unsigned word = (e & 3) == 0 ? w.x : (e & 3) == 1 ? w.y : (e & 3) == 2 ? w.z : w.w;
      signs[e] = (word >> 31) ? (int8_t)-1 : (int8_t)1;
    }
    if (e < l) {
      unsigned y = (unsigned)e;
      // at most span - m values >= m follow one another on a cycle
      for (int64_t it = 0; it <= span; ++it) {
        y = feistel(y, h, key);
        if ((int64_t)y < m) break;
      }
      rows[e] = (int32_t)y;
    }
  }
}

}  // namespace

curid_status srft_draw(const Ctx& ctx, int64_t m, int64_t l, uint64_t seed, int32_t* rows,
                       int8_t* signs) {
  if (m <= 0 || l <= 0) return CURID_OK;
  if (l > m || m > (1LL << 30)) return CURID_UNSUPPORTED;
  int h = 1;
  while ((1LL << (2 * h)) < m) ++h;
  const uint2 key = make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32));
  const unsigned blocks = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((m + 255) / 256, 16LL * ctx.num_sms));
  srft_draw_kernel<<<blocks, 256, 0, ctx.stream>>>(m, l, h, key, rows, signs);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template <typename real>
curid_status gaussian_fill(const Ctx& ctx, int64_t rows, int64_t cols, uint64_t seed, real* out,
                           int64_t ld) {
  const int64_t total = rows * cols;
  if (total <= 0) return CURID_OK;
  const uint2 key = make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32));
  const int64_t groups = (total + 3) / 4;
  const unsigned blocks = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((groups + 255) / 256, 16LL * ctx.num_sms));
  gaussian_kernel<real><<<blocks, 256, 0, ctx.stream>>>(total, cols, ld, key, out);
  CURID_LAUNCHED(ctx);
  return CURID_OK;
}

template curid_status gaussian_fill<float>(const Ctx&, int64_t, int64_t, uint64_t, float*,
                                           int64_t);
template curid_status gaussian_fill<double>(const Ctx&, int64_t, int64_t, uint64_t, double*,
                                            int64_t);

}  // namespace curid
