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
// round trip until the end.  The exchange (records, tags, pivot decision,
// pivot-column read, closing count exchange) lives in cpqr_exchange.cuh and
// is shared with the register-resident variant in cpqr_reg.cu, which
// cpqr_run launches instead when the slab fits in registers (at most 256
// rows, 128 in float64, and 64 columns per CTA).
// After the last step row i of S holds S1(i, c) for every original column c,
// J lists the pivots and then the unselected columns in ascending order.
#include <atomic>
#include <cstdlib>
#include <cstring>

#include "cpqr_exchange.cuh"

namespace curid {

namespace {

using namespace cpqr_x;

constexpr int kColsPerWarp = 4;  // columns a warp updates in one interleaved pass

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
    unsigned long long* dst = slot_of(P, bf, blockIdx.x);
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
  const int b = blockIdx.x;
  const int nc = P.nc, ldl = P.ldl, l = P.l;
  real* ys = reinterpret_cast<real*>(smem_raw);
  real* xv = ys + (int64_t)P.ncs * ldl;
  real* nrm = xv + ldl;
  int* active = reinterpret_cast<int*>(nrm + nc);

  __shared__ StepState<real> st;

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

  real normY = real(-1), nu_first = real(0);
  int k_eff = -1;
  int j = 0;
  for (;; ++j) {
    if (warp == 0) decide_pivot(P, j, normY, st);
    __syncthreads();
    if (st.stop) break;
    const int owner = st.owner, pcol = st.col;
    const real nu = st.nu;
    note_rank(P, j, nu, nu_first, k_eff);
    if (!fetch_pivot<kThreads>(P, j, owner, xv, st)) break;
    real beta, tau, scale;
    step_reflector(xv, j, nu, st, &beta, &tau, &scale);
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
  if (st.stop == 2) return;  // timed out: leave without further waits
  // S rows 0..k_done-1 in original column order
  for (int64_t e = tid; e < (int64_t)k_done * ncl; e += kThreads) {
    const int i = (int)(e / ncl), lc = (int)(e % ncl);
    P.S[(int64_t)i * P.lds + c0 + lc] =
        (!OV || lc < P.ncs) ? ys[(int64_t)lc * ldl + i] : slab_col<true>(P, ys, lc)[i];
  }
  finish_order(P, active, ncl, c0, k_done, k_eff, st);
}

template <typename real>
size_t cpqr_smem_bytes(int ncs, int nc, int ldl) {
  return (size_t)ncs * ldl * sizeof(real) + (size_t)ldl * sizeof(real) + (size_t)nc * sizeof(real) +
         (size_t)nc * sizeof(int) + 64;
}

// Grid, columns per CTA, how many of them fit in shared memory, and the warps
// per CTA of the register-resident kernel.
//
// One decomposition at a time (the handle's concurrency 1): one CTA per SM,
// the lowest latency per factorization.  With several in flight: the fewest
// CTAs whose registers hold the matrix (eight columns per warp).  The pivot
// exchange gets cheaper with fewer CTAs (records of 38-64 CTAs meet in about
// 2.4K cycles on GB300, of 152 in about twice that), the update gets longer,
// and the SMs left free run the other decompositions: the factorization
// takes about 1.2x as long on a third of the SMs.  Cooperative grids are
// gang-scheduled, so grids of concurrent factorizations queue whole.
// CURID_CPQR_CTAS in the environment overrides the choice for comparisons:
// "all" (one per SM) or "fewest".  (Eight-warp CTAs, two per SM, so that two
// concurrent factorizations share SMs, measured slower: 549/s against 613/s
// with four decompositions in flight.)
template <typename real>
curid_status cpqr_layout(const Ctx& ctx, int64_t l, int64_t n, int* G_out, int* nc_out,
                         int* ncs_out, int* warps_out = nullptr) {
  if (l <= 0 || n <= 0) return CURID_INVALID_ARG;
  const int gmax = std::min(ctx.num_sms, 32 * kMaxSlotsPerLane);
  int G = (int)std::min<int64_t>(gmax, n);
  int warps = 16;
  const char* env = std::getenv("CURID_CPQR_CTAS");
  bool fewest = ctx.concurrency > 1;
  if (env && std::strcmp(env, "all") == 0) fewest = false;
  if (env && std::strcmp(env, "fewest") == 0) fewest = true;
  if (fewest) {
    const int64_t rc = cpqr_reg_cols<real>((int)std::min<int64_t>(l, INT32_MAX), warps);
    if (rc > 0 && (n + rc - 1) / rc <= gmax) G = (int)((n + rc - 1) / rc);
  }
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
  if (warps_out) *warps_out = warps;
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
  s->slot_data = cv.take<unsigned long long>(2 * (size_t)G * slot_words<real>(l));
  s->counts = cv.take<int>(G);
  s->abort_flag = cv.take<int>(1);
  s->overflow = nc > ncs ? cv.take<real>((size_t)G * (nc - ncs) * (size_t)(l | 1)) : nullptr;
}

template <typename real>
curid_status cpqr_run(const Ctx& ctx, const real* Y, int64_t l, int64_t n, int64_t ldy, int k_max,
                      double tol, int32_t* J, real* S, int64_t lds, const CpqrScratch& s,
                      int which) {
  int G, nc, ncs, warps;
  CURID_TRY(cpqr_layout<real>(ctx, l, n, &G, &nc, &ncs, &warps));
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
  P.spin = ctx.spin;
  P.warps = warps;
  CURID_CUDA(cudaMemsetAsync(s.slots, 0, 2 * (size_t)G * sizeof(Rec), ctx.stream));
  CURID_CUDA(cudaMemsetAsync(s.abort_flag, 0, sizeof(int), ctx.stream));
  if (cpqr_reg_fits<real>(ctx, (int)l, nc, warps)) return cpqr_reg_launch<real>(ctx, P, G);
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
