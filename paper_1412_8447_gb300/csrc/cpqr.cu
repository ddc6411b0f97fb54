// Truncated column-pivoted Householder QR (Section 2.2, Eq. (2.4)-(2.5); the
// first line of Algorithms 1 and 4; the full-rank ID of C^* in Algorithm 2).
//
// GB300 design: one persistent CTA per SM (cooperative launch, so all CTAs
// are co-resident).  CTA b owns a contiguous slab of columns, held in shared
// memory for the whole factorization, column-major with an odd stride so a
// warp walking down a column is bank-conflict free.  A step j is:
//   1. warp 0 of every CTA reads the G candidate records of step j (one per
//      CTA: its largest residual column norm, that column's index, the sum
//      of its squared residual norms), all loads in flight together, and
//      picks the global pivot (largest norm, smallest index on ties) -- the
//      records double as the grid barrier;
//   2. every CTA reads the pivot column (rows j..l-1) that its owner
//      published and forms the same Householder reflector
//      H = I - tau v v^T (v(j) = 1), mapping it to beta e_j;
//   3. each warp applies H to one of the CTA's unselected columns and
//      recomputes that column's residual norm from rows j+1..l-1 (no norm
//      downdating, hence no cancellation to guard against);
//   4. warp 0 publishes the CTA's new local candidate for step j+1: the
//      record first, then the candidate column; every 64-bit word of both
//      carries the step's tag, so no fence is needed and a reader checks
//      each word for freshness.
// One grid-wide exchange and three CTA barriers per pivot step; no host
// round trip until the end.
// After the last step row i of S holds S1(i, c) for every original column c,
// J lists the pivots and then the unselected columns in ascending order.
#include <atomic>

#include "kernels.cuh"

namespace curid {

namespace {

// Exchange record of one CTA for one step: four 64-bit words, each
// (epoch << 32 | payload).  Every word carries the epoch, so a reader that
// sees the current epoch in all four has a consistent record no matter in
// which order the words became visible (each aligned 64-bit access is
// single-copy atomic).  Payloads: w0 = candidate column (kNoCol: none,
// kNonFinite: a non-finite norm was seen; the final exchange carries the
// CTA's count of unselected columns), w1/w2 = candidate norm (float bits in
// w1; float64 split high/low), w3 = sum of the CTA's squared residual norms
// as float (adaptive stop only).
struct alignas(128) Rec {  // one record per 128-byte line: no two writers share a line
  unsigned long long w[4];
  unsigned long long pad[12];
};

template <typename real>
struct CpqrParams {
  const real* Y;
  int64_t ldy;
  int l, n, k_max, nc, ldl;
  int ncs;                       // columns of a slab held in shared memory (the rest: gys)
  real* gys;                     // [G][nc - ncs][ldl] overflow columns, column-major
  real tol;
  real rank_rtol;
  int32_t* J;
  real* S;
  int64_t lds;
  Rec* recs;                     // [2][G]
  unsigned long long* slot_data;  // [2][G][l * words]: tagged candidate columns
  int* abort_flag;
  StatusBlock* status;
  int which;
  unsigned gen;                  // launch generation, high bits of every tag
};

// Published candidate columns are tagged word by word like the records, so a
// reader can tell a fresh element from a stale one without any fence on the
// writer's side: float32 -> one word (tag, bits); float64 -> two words
// (tag, high bits), (tag, low bits).  The tag of step e in launch g is
// (g << 20) | e.
template <typename real>
struct Words {
  static constexpr int W = sizeof(real) / 4;
};

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kColsPerWarp = 4;  // columns a warp updates in one interleaved pass
constexpr unsigned kNoCol = 0xffffffffu;
constexpr unsigned kNonFinite = 0xfffffffeu;
constexpr int kMaxSlotsPerLane = 5;  // G <= 160 (one CTA per SM; the GPU has 152)

__device__ __forceinline__ unsigned long long pack(unsigned epoch, unsigned payload) {
  return ((unsigned long long)epoch << 32) | payload;
}

__device__ __forceinline__ unsigned tag_of(unsigned gen, int epoch) {
  return (gen << 20) | (unsigned)epoch;
}

template <typename real>
__device__ __forceinline__ void put_tagged(unsigned long long* dst, unsigned tag, real v) {
  if (sizeof(real) == 8) {
    const unsigned long long b = (unsigned long long)__double_as_longlong((double)v);
    st_volatile_u64(dst, pack(tag, (unsigned)(b >> 32)));
    st_volatile_u64(dst + 1, pack(tag, (unsigned)(b & 0xffffffffull)));
  } else {
    st_volatile_u64(dst, pack(tag, __float_as_uint((float)v)));
  }
}

// Bounded read of one tagged element; false if it never became fresh.
template <typename real>
__device__ __forceinline__ bool get_tagged(const unsigned long long* src, unsigned tag, real* v,
                                           const int* abort_flag) {
  const long long t0 = clock64();
  while (true) {
    if (sizeof(real) == 8) {
      const unsigned long long a = ld_volatile_u64(src), b = ld_volatile_u64(src + 1);
      if ((unsigned)(a >> 32) == tag && (unsigned)(b >> 32) == tag) {
        *v = (real)__longlong_as_double((long long)(((a & 0xffffffffull) << 32) |
                                                     (b & 0xffffffffull)));
        return true;
      }
    } else {
      const unsigned long long a = ld_volatile_u64(src);
      if ((unsigned)(a >> 32) == tag) {
        *v = (real)__uint_as_float((unsigned)(a & 0xffffffffull));
        return true;
      }
    }
    if (ld_volatile_i32(abort_flag) || clock64() - t0 > kSpinBudget) return false;
  }
}

template <typename real>
__device__ __forceinline__ void norm_words(real v, unsigned* hi, unsigned* lo) {
  if (sizeof(real) == 8) {
    const unsigned long long b = (unsigned long long)__double_as_longlong((double)v);
    *hi = (unsigned)(b >> 32);
    *lo = (unsigned)(b & 0xffffffffull);
  } else {
    *hi = __float_as_uint((float)v);
    *lo = 0u;
  }
}

template <typename real>
__device__ __forceinline__ real words_norm(unsigned hi, unsigned lo) {
  if (sizeof(real) == 8)
    return (real)__longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
  return (real)__uint_as_float(hi);
}

__device__ __forceinline__ void st_rec(Rec* r, unsigned long long a, unsigned long long b,
                                       unsigned long long c, unsigned long long d) {
  asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(&r->w[0]), "l"(a), "l"(b)
               : "memory");
  asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(&r->w[2]), "l"(c), "l"(d)
               : "memory");
}

__device__ __forceinline__ void ld_rec(const Rec* r, unsigned long long* w) {
  asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];"
               : "=l"(w[0]), "=l"(w[1])
               : "l"(&r->w[0]));
  asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];"
               : "=l"(w[2]), "=l"(w[3])
               : "l"(&r->w[2]));
}

template <typename real>
__device__ __forceinline__ bool better(real na, unsigned ca, real nb, unsigned cb) {
  // (na, ca) beats (nb, cb): larger norm, then smaller column; kNoCol loses.
  if (ca == kNoCol) return false;
  if (cb == kNoCol) return true;
  if (na > nb) return true;
  if (na < nb) return false;
  return ca < cb;
}

// Warp 0: wait until all G records of buffer `bf` carry `epoch`, keeping
// their words.  Each lane polls up to kMaxSlotsPerLane records with all of
// its loads in flight at once.  Returns false on timeout or abort.
template <typename real>
__device__ bool gather_records(const CpqrParams<real>& P, int bf, unsigned epoch,
                               unsigned long long (*w)[4]) {
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x;
  const Rec* base = P.recs + (size_t)bf * G;
  // float32 without a tolerance needs only (column, norm): one 16-byte load
  const bool full = sizeof(real) == 8 || P.tol > real(0);
  unsigned pending = 0;
#pragma unroll
  for (int r = 0; r < kMaxSlotsPerLane; ++r)
    if (lane + 32 * r < G) pending |= 1u << r;
  bool ok = true;
  const long long t0 = clock64();
  for (int round = 0; pending; ++round) {
#pragma unroll
    for (int r = 0; r < kMaxSlotsPerLane; ++r) {
      if (!(pending & (1u << r))) continue;
      const Rec* rec = base + lane + 32 * r;
      if (full) {
        ld_rec(rec, w[r]);
      } else {
        asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];"
                     : "=l"(w[r][0]), "=l"(w[r][1])
                     : "l"(&rec->w[0]));
        w[r][2] = w[r][3] = (unsigned long long)epoch << 32;
      }
    }
#pragma unroll
    for (int r = 0; r < kMaxSlotsPerLane; ++r) {
      if (!(pending & (1u << r))) continue;
      bool fresh = true;
#pragma unroll
      for (int q = 0; q < 4; ++q) fresh &= (unsigned)(w[r][q] >> 32) == epoch;
      if (fresh) pending &= ~(1u << r);
    }
    if (!pending) break;
    if ((round & 15) == 15) {
      if (ld_volatile_i32(P.abort_flag)) { ok = false; break; }
      if (clock64() - t0 > kSpinBudget) {
        atomicExch(P.abort_flag, 1);
        ok = false;
        break;
      }
    }
  }
  ok = __all_sync(0xffffffffu, ok);
  return ok;
}

// Column lc of this CTA's slab: shared memory for lc < ncs, else the CTA's
// part of the global overflow area (same column-major layout).
template <bool OV, typename real>
__device__ __forceinline__ real* slab_col(const CpqrParams<real>& P, real* ys, int lc) {
  if constexpr (!OV) return ys + (int64_t)lc * P.ldl;
  return lc < P.ncs ? ys + (int64_t)lc * P.ldl
                    : P.gys + ((int64_t)blockIdx.x * (P.nc - P.ncs) + (lc - P.ncs)) * P.ldl;
}

// Warp 0: pick the CTA's candidate (largest residual norm among its
// unselected columns, smallest index on ties), publish the record of `epoch`
// in buffer `bf`, then copy the candidate's rows r0..l-1 to the CTA's data
// slot (tagged words; a reader waits for the fresh tag of each word).
template <bool OV, typename real>
__device__ void publish(const CpqrParams<real>& P, real* ys, const real* nrm,
                        const int* active, int ncl, int c0, int r0, int bf, unsigned epoch) {
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x;
  real bn = real(-1), ss = real(0);
  int bi = -1, nf = 0;
  for (int lc = lane; lc < ncl; lc += 32) {
    if (!active[lc]) continue;
    const real v = nrm[lc];
    if (!isfinite(v)) nf = 1;
    ss += v * v;
    if (bi < 0 || v > bn) { bn = v; bi = lc; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const real on = __shfl_xor_sync(0xffffffffu, bn, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi >= 0 && (bi < 0 || on > bn || (on == bn && oi < bi))) { bn = on; bi = oi; }
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    nf |= __shfl_xor_sync(0xffffffffu, nf, o);
  }
  const unsigned tag = tag_of(P.gen, (int)epoch);
  // the record first: readers validate every word of the column by its tag,
  // so the column copy below overlaps the record's way to the other CTAs
  if (lane == 0) {
    unsigned hi, lo;
    norm_words<real>(bi >= 0 ? bn : real(0), &hi, &lo);
    const unsigned col = nf ? kNonFinite : (bi >= 0 ? (unsigned)(c0 + bi) : kNoCol);
    st_rec(P.recs + (size_t)bf * G + blockIdx.x, pack(tag, col), pack(tag, hi), pack(tag, lo),
           pack(tag, __float_as_uint((float)ss)));
  }
  if (bi >= 0 && !nf) {
    constexpr int W = Words<real>::W;
    unsigned long long* dst = P.slot_data + ((int64_t)bf * G + blockIdx.x) * P.l * W;
    if (!OV || bi < P.ncs) {
      const real* src = ys + (int64_t)bi * P.ldl;
      for (int r = r0 + lane; r < P.l; r += 32) put_tagged<real>(dst + (int64_t)r * W, tag, src[r]);
    } else {
      const real* src = slab_col<OV>(P, ys, bi);
      for (int r = r0 + lane; r < P.l; r += 32) put_tagged<real>(dst + (int64_t)r * W, tag, src[r]);
    }
  }
}

// One interleaved pass of a warp over columns base, base + kWarps, ... of
// its slab (see the step loop).  SH: all of them are in shared memory, so
// their pointers come straight from the shared array and the accesses
// compile to shared-memory loads and stores.
template <bool SH, typename real>
__device__ __forceinline__ void update_group(const CpqrParams<real>& P, real* ys, const real* xv,
                                             real* nrm, int* active, int ncl, int c0, int j,
                                             int pcol, real beta, real tau, real scale, int base,
                                             int lane) {
  const int l = P.l;
  bool v[kColsPerWarp];
  real* y[kColsPerWarp];
#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c) {
    const int lc = base + c * kWarps;
    v[c] = lc < ncl && active[lc] != 0;
    y[c] = SH ? ys + (int64_t)(lc < ncl ? lc : base) * P.ldl
              : slab_col<true>(P, ys, lc < ncl ? lc : base);
    if (v[c] && c0 + lc == pcol) {
      for (int r = j + lane; r < l; r += 32) y[c][r] = r == j ? beta : real(0);
      if (lane == 0) {
        active[lc] = 0;
        P.J[j] = pcol;
      }
      v[c] = false;
    }
  }
  bool any = false;
#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c) any |= v[c];
  if (!any) return;
  constexpr int RB = sizeof(real) == 4 ? 4 : 2;  // rows per lane held in registers
  real d[kColsPerWarp];
#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c) d[c] = real(0);
  real wj[kColsPerWarp], ws[kColsPerWarp], q[kColsPerWarp];
  if (l - j - 1 <= 32 * RB) {
    // every row this lane touches fits in registers: one load of the
    // column part, dot products, reflector update and new norms from the
    // registers, one store
    real xr[RB], yr[kColsPerWarp][RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int r = j + 1 + lane + 32 * u;
      const bool ok = r < l;
      xr[u] = ok ? xv[r] : real(0);
#pragma unroll
      for (int c = 0; c < kColsPerWarp; ++c) yr[c][u] = (ok && v[c]) ? y[c][r] : real(0);
    }
#pragma unroll
    for (int u = 0; u < RB; ++u)
#pragma unroll
      for (int c = 0; c < kColsPerWarp; ++c) d[c] += xr[u] * yr[c][u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < kColsPerWarp; ++c) d[c] += __shfl_xor_sync(0xffffffffu, d[c], o);
#pragma unroll
    for (int c = 0; c < kColsPerWarp; ++c) {
      wj[c] = v[c] ? tau * (y[c][j] + scale * d[c]) : real(0);
      ws[c] = wj[c] * scale;
      q[c] = real(0);
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < kColsPerWarp; ++c)
        if (v[c]) y[c][j] -= wj[c];
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int r = j + 1 + lane + 32 * u;
#pragma unroll
      for (int c = 0; c < kColsPerWarp; ++c) {
        const real nv = yr[c][u] - ws[c] * xr[u];
        q[c] += nv * nv;  // rows past l hold zeros
        if (v[c] && r < l) y[c][r] = nv;
      }
    }
  } else {
    for (int r = j + 1 + lane; r < l; r += 32) {
      const real x = xv[r];
#pragma unroll
      for (int c = 0; c < kColsPerWarp; ++c)
        if (v[c]) d[c] += x * y[c][r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < kColsPerWarp; ++c) d[c] += __shfl_xor_sync(0xffffffffu, d[c], o);
#pragma unroll
    for (int c = 0; c < kColsPerWarp; ++c) {
      wj[c] = v[c] ? tau * (y[c][j] + scale * d[c]) : real(0);
      ws[c] = wj[c] * scale;
      q[c] = real(0);
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < kColsPerWarp; ++c)
        if (v[c]) y[c][j] -= wj[c];
    }
    for (int r = j + 1 + lane; r < l; r += 32) {
      const real x = xv[r];
#pragma unroll
      for (int c = 0; c < kColsPerWarp; ++c) {
        if (!v[c]) continue;
        const real nv = y[c][r] - ws[c] * x;
        y[c][r] = nv;
        q[c] += nv * nv;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < kColsPerWarp; ++c) q[c] += __shfl_xor_sync(0xffffffffu, q[c], o);
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < kColsPerWarp; ++c)
      if (v[c]) nrm[base + c * kWarps] = sqrt(q[c]);
  }
}

template <typename real, bool OV>
__global__ void __launch_bounds__(kThreads, 1) cpqr_kernel(CpqrParams<real> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x, b = blockIdx.x;
  const int nc = P.nc, ldl = P.ldl, l = P.l;
  real* ys = reinterpret_cast<real*>(smem_raw);
  real* xv = ys + (int64_t)P.ncs * ldl;
  real* nrm = xv + ldl;
  int* active = reinterpret_cast<int*>(nrm + nc);

  __shared__ int s_stop, s_owner, s_col, s_prefix;
  __shared__ real s_nu;

  const int c0 = b * nc;
  const int ncl = max(0, min(nc, P.n - c0));

  // load the slab, column-major in shared memory
  for (int64_t e = tid; e < (int64_t)l * ncl; e += kThreads) {
    const int r = (int)(e / ncl), lc = (int)(e % ncl);
    const real yv = P.Y[(int64_t)r * P.ldy + c0 + lc];
    if (!OV || lc < P.ncs) ys[(int64_t)lc * ldl + r] = yv;
    else slab_col<true>(P, ys, lc)[r] = yv;
  }
  for (int lc = tid; lc < nc; lc += kThreads) active[lc] = lc < ncl ? 1 : 0;
  __syncthreads();
  for (int lc = warp; lc < ncl; lc += kWarps) {
    real s2 = real(0);
    if (!OV || lc < P.ncs) {
      const real* y = ys + (int64_t)lc * ldl;
      for (int r = lane; r < l; r += 32) s2 += y[r] * y[r];
    } else {
      const real* y = slab_col<true>(P, ys, lc);
      for (int r = lane; r < l; r += 32) s2 += y[r] * y[r];
    }
    s2 = warp_sum(s2);
    if (lane == 0) nrm[lc] = sqrt(s2);
  }
  __syncthreads();
  if (warp == 0) publish<OV>(P, ys, nrm, active, ncl, c0, 0, 0, 1u);
  __shared__ int s_stale;

  real normY = real(-1), nu_first = real(0);
  int k_eff = -1;
  int j = 0;
  for (;; ++j) {
    const int bf = j & 1;
    if (warp == 0) {
      unsigned long long w[kMaxSlotsPerLane][4];
      const bool ok = gather_records(P, bf, tag_of(P.gen, j + 1), w);
      // global pivot and totals, identical in every CTA
      real bn = real(-1), tot = real(0);
      unsigned bc = kNoCol;
      int bo = -1, nf = 0;
      if (ok) {
#pragma unroll
        for (int r = 0; r < kMaxSlotsPerLane; ++r) {
          const int s = lane + 32 * r;
          if (s >= G) continue;
          const unsigned col = (unsigned)(w[r][0] & 0xffffffffull);
          const real nn = words_norm<real>((unsigned)(w[r][1] & 0xffffffffull),
                                           (unsigned)(w[r][2] & 0xffffffffull));
          tot += (real)__uint_as_float((unsigned)(w[r][3] & 0xffffffffull));
          if (col == kNonFinite) nf = 1;
          else if (better(nn, col, bn, bc)) { bn = nn; bc = col; bo = s; }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const real on = __shfl_xor_sync(0xffffffffu, bn, o);
        const unsigned oc = __shfl_xor_sync(0xffffffffu, bc, o);
        const int oo = __shfl_xor_sync(0xffffffffu, bo, o);
        if (better(on, oc, bn, bc)) { bn = on; bc = oc; bo = oo; }
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        nf |= __shfl_xor_sync(0xffffffffu, nf, o);
      }
      if (lane == 0) {
        int stop = 0;
        if (!ok) {
          stop = 2;
          set_flag(&P.status->flags, FLAG_TIMEOUT);
        } else if (nf) {
          stop = 1;
          if (b == 0) set_flag(&P.status->flags, FLAG_NONFINITE);
        } else if (j >= P.k_max || bc == kNoCol) {
          stop = 1;
        } else {
          if (normY < real(0)) normY = sqrt(tot);
          if (P.tol > real(0) && sqrt(tot) <= P.tol * normY) stop = 1;
        }
        s_stop = stop;
        s_owner = bo;
        s_col = (int)bc;
        s_nu = bn;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int owner = s_owner, pcol = s_col;
    const real nu = s_nu;
    if (j == 0) nu_first = nu;
    if (k_eff < 0 && (nu == real(0) || nu <= P.rank_rtol * nu_first)) {
      k_eff = j;
      if (b == 0 && tid == 0) set_flag(&P.status->flags, FLAG_RANK_DEFICIENT);
    }
    // pivot column rows j..l-1, as its owner published it (tagged words)
    {
      constexpr int W = Words<real>::W;
      const unsigned long long* src = P.slot_data + ((int64_t)bf * G + owner) * l * W;
      const unsigned tag = tag_of(P.gen, j + 1);
      if (tid == 0) s_stale = 0;
      __syncthreads();
      for (int r = j + tid; r < l; r += kThreads) {
        real v;
        if (!get_tagged<real>(src + (int64_t)r * W, tag, &v, P.abort_flag)) {
          s_stale = 1;
          v = real(0);
        }
        xv[r] = v;
      }
      __syncthreads();
      if (s_stale) {
        if (tid == 0) {
          atomicExch(P.abort_flag, 1);
          set_flag(&P.status->flags, FLAG_TIMEOUT);
        }
        s_stop = 2;
        break;
      }
    }
    // Householder reflector H = I - tau v v^T with v(j) = 1, v(r) = scale x(r):
    // H x = beta e_j, beta = -sign(alpha) nu
    const real alpha = xv[j];
    const real beta = alpha >= real(0) ? -nu : nu;
    real tau = real(0), scale = real(0);
    if (nu > real(0)) {
      tau = (beta - alpha) / beta;
      scale = real(1) / (alpha - beta);
    }
    // apply H to every unselected local column, recompute its residual norm
    // from rows j+1..l-1; the owner retires the pivot column.  Warp w owns
    // columns w, w + 16, w + 32, w + 48 and updates them in one interleaved
    // pass so their reductions overlap.
    for (int base = warp; base < ncl; base += kColsPerWarp * kWarps) {
      // columns past ncl are unused (their pointer falls back to column base)
      if (!OV || min(ncl - 1, base + (kColsPerWarp - 1) * kWarps) < P.ncs)
        update_group<true>(P, ys, xv, nrm, active, ncl, c0, j, pcol, beta, tau, scale, base, lane);
      else
        update_group<false>(P, ys, xv, nrm, active, ncl, c0, j, pcol, beta, tau, scale, base, lane);
    }
    __syncthreads();
    if (warp == 0) publish<OV>(P, ys, nrm, active, ncl, c0, j + 1, (j + 1) & 1, (unsigned)(j + 2));

  }
  const int k_done = j;
  if (s_stop == 2) return;  // timed out: leave without further waits
  // S rows 0..k_done-1 in original column order
  for (int64_t e = tid; e < (int64_t)k_done * ncl; e += kThreads) {
    const int i = (int)(e / ncl), lc = (int)(e % ncl);
    P.S[(int64_t)i * P.lds + c0 + lc] =
        (!OV || lc < P.ncs) ? ys[(int64_t)lc * ldl + i] : slab_col<true>(P, ys, lc)[i];
  }
  // unselected columns in ascending order after the pivots: exchange counts
  const int fbf = (j + 1) & 1;
  const unsigned fep = tag_of(P.gen, j + 2);
  if (warp == 0) {
    int cnt = 0;
    for (int lc = lane; lc < ncl; lc += 32) cnt += active[lc];
    cnt = warp_sum(cnt);
    if (lane == 0) {
      st_rec(P.recs + (size_t)fbf * G + b, pack(fep, (unsigned)cnt), pack(fep, 0u), pack(fep, 0u),
             pack(fep, 0u));
    }
    unsigned long long w[kMaxSlotsPerLane][4];
    const bool ok = gather_records(P, fbf, fep, w);
    int pre = 0;
    if (ok) {
#pragma unroll
      for (int r = 0; r < kMaxSlotsPerLane; ++r)
        if (lane + 32 * r < b) pre += (int)(w[r][0] & 0xffffffffull);
    }
    pre = warp_sum(pre);
    if (lane == 0) {
      s_prefix = pre;
      s_stop = ok ? 0 : 2;
      if (!ok) set_flag(&P.status->flags, FLAG_TIMEOUT);
    }
  }
  __syncthreads();
  if (s_stop) return;
  if (tid == 0) {
    int pos = k_done + s_prefix;
    for (int lc = 0; lc < ncl; ++lc)
      if (active[lc]) P.J[pos++] = c0 + lc;
    if (b == 0) {
      if (P.which == 0) {
        P.status->k_done = k_done;
        P.status->k_eff = k_eff < 0 ? k_done : k_eff;
      } else {
        P.status->k_row = k_eff < 0 ? k_done : k_eff;
      }
    }
  }
}

template <typename real>
size_t cpqr_smem_bytes(int ncs, int nc, int ldl) {
  return (size_t)ncs * ldl * sizeof(real) + (size_t)ldl * sizeof(real) + (size_t)nc * sizeof(real) +
         (size_t)nc * sizeof(int) + 64;
}

// Grid, columns per CTA and how many of them fit in shared memory.
template <typename real>
curid_status cpqr_layout(const Ctx& ctx, int64_t l, int64_t n, int* G_out, int* nc_out,
                         int* ncs_out) {
  if (l <= 0 || n <= 0) return CURID_INVALID_ARG;
  int G = (int)std::min<int64_t>(std::min(ctx.num_sms, 32 * kMaxSlotsPerLane), n);
  const int nc = (int)((n + G - 1) / G);
  G = (int)((n + nc - 1) / nc);
  const int ldl = (int)(l | 1);
  // the kernel's static shared variables share the per-block limit
  const size_t fixed = cpqr_smem_bytes<real>(0, nc, ldl) + 1024;
  if (fixed > ctx.smem_optin) return CURID_UNSUPPORTED;
  const int ncs = (int)std::min<size_t>(nc, (ctx.smem_optin - fixed) / ((size_t)ldl * sizeof(real)));
  *G_out = G;
  *nc_out = nc;
  *ncs_out = ncs;
  return CURID_OK;
}

}  // namespace

template <typename real>
curid_status cpqr_plan(const Ctx& ctx, int64_t l, int64_t n, int* grid, size_t* smem) {
  int G, nc, ncs;
  CURID_TRY(cpqr_layout<real>(ctx, l, n, &G, &nc, &ncs));
  *grid = G;
  *smem = cpqr_smem_bytes<real>(ncs, nc, (int)(l | 1));
  return CURID_OK;
}

template <typename real>
void cpqr_carve(Carver& cv, const Ctx& ctx, int64_t l, int64_t n, CpqrScratch* s) {
  int G = 1, nc = 1, ncs = 1;
  if (cpqr_layout<real>(ctx, l, n, &G, &nc, &ncs) != CURID_OK) G = nc = ncs = 1;
  s->grid = G;
  s->slots = cv.take<Rec>(2 * (size_t)G);
  s->slot_data = cv.take<unsigned long long>(2 * (size_t)G * l * Words<real>::W);
  s->counts = cv.take<int>(G);
  s->abort_flag = cv.take<int>(1);
  s->overflow = nc > ncs ? cv.take<real>((size_t)G * (nc - ncs) * (size_t)(l | 1)) : nullptr;
}

template <typename real>
curid_status cpqr_run(const Ctx& ctx, const real* Y, int64_t l, int64_t n, int64_t ldy, int k_max,
                      double tol, int32_t* J, real* S, int64_t lds, const CpqrScratch& s,
                      int which) {
  int G, nc, ncs;
  CURID_TRY(cpqr_layout<real>(ctx, l, n, &G, &nc, &ncs));
  if (G != s.grid || (nc > ncs && !s.overflow)) return CURID_INVALID_ARG;
  const size_t smem = cpqr_smem_bytes<real>(ncs, nc, (int)(l | 1));
  CpqrParams<real> P;
  P.Y = Y;
  P.ldy = ldy;
  P.l = (int)l;
  P.n = (int)n;
  P.k_max = k_max;
  P.nc = nc;
  P.ncs = ncs;
  P.gys = static_cast<real*>(s.overflow);
  P.ldl = (int)(l | 1);
  P.tol = (real)tol;
  // a pivot norm at or below 2 sqrt(l) eps nu_1 is rounding noise (Section 2.3's
  // singular S11): k_eff stops there
  P.rank_rtol = real(2) * (real)std::sqrt((double)l) *
                (sizeof(real) == 8 ? (real)2.220446049250313e-16 : (real)1.1920929e-07);
  P.J = J;
  P.S = S;
  P.lds = lds;
  P.recs = static_cast<Rec*>(s.slots);
  P.slot_data = static_cast<unsigned long long*>(s.slot_data);
  static std::atomic<unsigned> generation{0};
  P.gen = (generation.fetch_add(1) + 1) & 0xfffu;
  P.abort_flag = s.abort_flag;
  P.status = ctx.status;
  P.which = which;
  CURID_CUDA(cudaMemsetAsync(s.slots, 0, 2 * (size_t)G * sizeof(Rec), ctx.stream));
  CURID_CUDA(cudaMemsetAsync(s.abort_flag, 0, sizeof(int), ctx.stream));
  auto fn = nc > ncs ? cpqr_kernel<real, true> : cpqr_kernel<real, false>;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  void* args[] = {&P};
  CURID_CUDA(cudaLaunchCooperativeKernel((void*)fn, dim3(G), dim3(kThreads), args, smem,
                                         ctx.stream));
  if (ctx.launches) ++*ctx.launches;
  return CURID_OK;
}

template curid_status cpqr_plan<float>(const Ctx&, int64_t, int64_t, int*, size_t*);
template curid_status cpqr_plan<double>(const Ctx&, int64_t, int64_t, int*, size_t*);
template void cpqr_carve<float>(Carver&, const Ctx&, int64_t, int64_t, CpqrScratch*);
template void cpqr_carve<double>(Carver&, const Ctx&, int64_t, int64_t, CpqrScratch*);
template curid_status cpqr_run<float>(const Ctx&, const float*, int64_t, int64_t, int64_t, int,
                                      double, int32_t*, float*, int64_t, const CpqrScratch&, int);
template curid_status cpqr_run<double>(const Ctx&, const double*, int64_t, int64_t, int64_t, int,
                                       double, int32_t*, double*, int64_t, const CpqrScratch&,
                                       int);

}  // namespace curid
