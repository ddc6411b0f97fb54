// Truncated column-pivoted Householder QR (Section 2.2, Eq. (2.4)-(2.5); the
// first line of Algorithms 1 and 4; the full-rank ID of C^* in Algorithm 2).
//
// GB300 design: one persistent CTA per SM (cooperative launch, so all CTAs
// are co-resident).  CTA b owns a contiguous slab of columns for the whole
// factorization, cut into groups of four neighbouring columns stored row by
// row: one 16-byte vector holds the four columns of a row in float32, so a
// warp reads or writes a group's rows with one vector access per lane and 32
// lanes on 32 consecutive rows touch 512 contiguous bytes (no bank
// conflicts at any row count).  In float32 warps 1..15 each keep one group
// in their registers (lane t holds rows t, t + 32, ...; up to 544 rows), the
// other groups live in shared memory, and groups beyond shared memory in a
// global overflow area of the same layout: registers and shared memory
// together hold about 360 KB per SM, the 20000 columns of 520 rows of the
// 20000 x 20000 randomized CUR on 152 SMs without overflow.  Warp 0 gathers
// the pivot records and holds no register group (no warp carries both the
// records in flight and a register group: 128 registers per thread, no
// spills); it takes two memory groups in its place.
// A step j is:
//   1. warp 0 of every CTA reads the G candidate records of step j (one per
//      CTA: its largest residual column norm, that column's index, the sum
//      of its squared residual norms), all loads in flight together, and
//      picks the global pivot (largest norm, smallest index on ties) -- the
//      records double as the grid barrier;
//   2. every CTA reads the pivot column (rows j..l-1) that its owner
//      published and forms the same Householder reflector
//      H = I - tau v v^T (v(j) = 1, v(r) = scale x(r) below row j), mapping
//      it to beta e_j;
//   3. each warp applies H to its groups: the four dot products of a group
//      are summed by one transpose-and-reduce butterfly, the update touches
//      rows j..l-1 only, and the residual norms are recomputed from rows
//      j+1..l-1 (no norm downdating, hence no cancellation to guard
//      against); the warp holding the pivot column retires it (beta at row
//      j, zeros below) and every warp posts its best unselected column;
//   4. warp 0 publishes the CTA's record for step j+1 and the warp holding
//      the CTA's best column copies it to the CTA's slot; every 64-bit word
//      of both carries the step's tag, so no fence is needed and a reader
//      checks each word for freshness.
// One grid-wide exchange and three CTA barriers per pivot step; no host
// round trip until the end.  The exchange (records, tags, pivot decision,
// pivot-column read, closing count exchange) lives in cpqr_exchange.cuh and
// is shared with the register-resident variant in cpqr_reg.cu, which
// cpqr_run launches instead when the whole slab fits in registers (at most
// 256 rows, 128 in float64, and 64 or 128 columns per CTA).
// After the last step row i of S holds S1(i, c) for every original column c,
// J lists the pivots and then the unselected columns in ascending order.
#include <atomic>
#include <cstdlib>
#include <cstring>

#include "cpqr_exchange.cuh"

namespace curid {

namespace {

using namespace cpqr_x;

// Rows per lane of the register-resident groups (float32 only: four columns
// of 17 rows are 68 registers): matrices of up to 544 rows; up to 224 rows
// take 7 rows per lane, so no register row block lies past the matrix.
constexpr int kGroupRegRows = 17;
constexpr int kGroupRegRowsShort = 7;

template <typename real>
constexpr int group_reg_rows(int64_t l) {
  if (sizeof(real) != 4) return 0;
  if (l <= 32 * kGroupRegRowsShort) return kGroupRegRowsShort;
  return l <= 32 * kGroupRegRows ? kGroupRegRows : 0;
}

// Four neighbouring columns of one row.
template <typename real>
struct alignas(4 * sizeof(real)) Quad {
  real x, y, z, w;
};

template <typename real>
__device__ __forceinline__ Quad<real> ldq(const Quad<real>* p) {
  if constexpr (sizeof(real) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    return {t.x, t.y, t.z, t.w};
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    return {a.x, a.y, b.x, b.y};
  }
}

template <typename real>
__device__ __forceinline__ void stq(Quad<real>* p, const Quad<real>& q) {
  if constexpr (sizeof(real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(q.x, q.y, q.z, q.w);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(q.x, q.y);
    reinterpret_cast<double2*>(p)[1] = make_double2(q.z, q.w);
  }
}

// Component c of q, c known only at run time (selects, no local memory).
template <typename real>
__device__ __forceinline__ real comp(const Quad<real>& q, int c) {
  return c == 0 ? q.x : c == 1 ? q.y : c == 2 ? q.z : q.w;
}

template <typename real>
__device__ __forceinline__ void set_comp(Quad<real>& q, int c, real v) {
  if (c == 0) q.x = v;
  else if (c == 1) q.y = v;
  else if (c == 2) q.z = v;
  else q.w = v;
}

// Unselected columns of group g as a 4-bit mask.
__device__ __forceinline__ unsigned act_of(const int* active, int g) {
  const int4 a = *reinterpret_cast<const int4*>(active + 4 * g);
  return (a.x ? 1u : 0u) | (a.y ? 2u : 0u) | (a.z ? 4u : 0u) | (a.w ? 8u : 0u);
}

// Rows of group g >= NR (NR: register groups per CTA): shared memory for the
// first P.ncs, then the CTA's part of the global overflow area.
template <int NR, bool OV, typename real>
__device__ __forceinline__ Quad<real>* group_rows(const CpqrParams<real>& P, Quad<real>* ys, int g) {
  const int s = g - NR;
  if (!OV || s < P.ncs) return ys + (int64_t)s * P.l;
  const int ngo = P.nc / 4 - NR - P.ncs;
  return reinterpret_cast<Quad<real>*>(P.gys) + ((int64_t)blockIdx.x * ngo + (s - P.ncs)) * P.l;
}

// A lane's running best over the columns it sees: after reduce4 the lanes of
// one eighth of the warp hold the same column, so the warp's best is merged
// over the lanes 8 and 16 apart only.  Columns are compared by their squared
// residual norms (the same order); the square root is taken once, for the
// CTA's record.
template <typename real>
struct LaneBest {
  real bn, ss;  // best squared norm, sum of squared norms
  int bi, nf;
  __device__ __forceinline__ void reset() {
    bn = real(-1);
    ss = real(0);
    bi = -1;
    nf = 0;
  }
  // an unselected local column lc with squared residual norm q2
  __device__ __forceinline__ void add(real q2, int lc) {
    ss += q2;
    if (!isfinite(q2)) nf = 1;
    else if (local_better(q2, lc, bn, bi)) {
      bn = q2;
      bi = lc;
    }
  }
};

template <typename real>
__device__ __forceinline__ void post_best(LaneBest<real> b, int lane, int warp, WarpBest<real>& wb) {
#pragma unroll
  for (int o = 8; o <= 16; o <<= 1) {
    const real on = __shfl_xor_sync(0xffffffffu, b.bn, o);
    const int oi = __shfl_xor_sync(0xffffffffu, b.bi, o);
    if (local_better(on, oi, b.bn, b.bi)) {
      b.bn = on;
      b.bi = oi;
    }
    b.ss += __shfl_xor_sync(0xffffffffu, b.ss, o);
    b.nf |= __shfl_xor_sync(0xffffffffu, b.nf, o);
  }
  if (lane == 0) {
    wb.bn[warp] = b.bn;
    wb.bi[warp] = b.bi;
    wb.ss[warp] = b.ss;
    wb.nf[warp] = b.nf;
  }
}

// Owner warp of group g.  With register groups (NR = 15): group g < 15 is
// the register group of warp g + 1; memory group m = g - 15 belongs to warp
// 0 for m = 0, 1 and then to warps 1, 2, ..., 15, 0, 1, ... in turn: warp 0,
// which gathers the records and holds no register group, takes two memory
// groups in its place (a register group costs about as much as two).
// Without register groups: warp (g + 1) mod 16.
template <int NR>
__device__ __forceinline__ int group_owner(int g) {
  if (NR == 0) return (g + 1) % kWarps;
  if (g < NR) return g + 1;
  const int m = g - NR;
  return m < 2 ? 0 : (m - 1) % kWarps;
}

// A warp's memory groups in the order it updates them: first, next.
template <int NR>
__device__ __forceinline__ int first_mem_group(int warp) {
  return NR == 0 ? (warp + kWarps - 1) % kWarps : NR + (warp ? warp + 1 : 0);
}
template <int NR>
__device__ __forceinline__ int next_mem_group(int g) {
  return (NR > 0 && g == NR) ? NR + 1 : g + kWarps;
}

// Every warp, after the barrier that follows post_best (wb holds squared
// norms): the CTA's candidate for epoch `epoch`.  Warp 0 publishes the
// record in buffer bf; the warp that owns the candidate's group copies its
// rows r0..l-1 to the CTA's data slot
// as tagged words, from its registers or from the group's rows (readers check
// every word's tag, so the two writes need no order between them).
template <int RPL, bool REGS, int NR, bool OV, typename real>
__device__ __forceinline__ void publish(const CpqrParams<real>& P, Quad<real>* ys,
                                        const WarpBest<real>& wb, const Quad<real> (&yr)[RPL],
                                        int c0, int r0, int bf, unsigned epoch, int lane,
                                        int warp) {
  real bn = lane < kWarps ? wb.bn[lane] : real(-1);
  int bi = lane < kWarps ? wb.bi[lane] : -1;
  int nf = lane < kWarps ? wb.nf[lane] : 0;
#pragma unroll
  for (int o = 1; o < kWarps; o <<= 1) {
    const real on = __shfl_xor_sync(0xffffffffu, bn, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (local_better(on, oi, bn, bi)) {
      bn = on;
      bi = oi;
    }
    nf |= __shfl_xor_sync(0xffffffffu, nf, o);
  }
  // lanes 0..15 agree; take lane 0's view everywhere
  bn = __shfl_sync(0xffffffffu, bn, 0);
  bi = __shfl_sync(0xffffffffu, bi, 0);
  nf = __shfl_sync(0xffffffffu, nf, 0);
  const unsigned tag = tag_of(P.gen, (int)epoch);
  if (warp == 0) {
    real ss = lane < kWarps ? wb.ss[lane] : real(0);
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) {
      unsigned hi, lo;
      norm_words<real>(bi >= 0 ? sqrt(bn) : real(0), &hi, &lo);
      const unsigned col = nf ? kNonFinite : (bi >= 0 ? (unsigned)(c0 + bi) : kNoCol);
      st_rec(P.recs + (size_t)bf * gridDim.x + blockIdx.x, pack(tag, col), pack(tag, hi),
             pack(tag, lo), pack(tag, __float_as_uint((float)ss)));
    }
  }
  if (bi < 0 || nf || group_owner<NR>(bi >> 2) != warp) return;
  constexpr int W = Words<real>::W;
  unsigned long long* dst = slot_of(P, bf, blockIdx.x);
  const int g = bi >> 2, c = bi & 3;
  if (REGS && g < NR) {
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      const int r = lane + 32 * u;
      if (r >= r0 && r < P.l) put_tagged<real>(dst + (int64_t)r * W, tag, comp(yr[u], c));
    }
  } else {
    const real* src = reinterpret_cast<const real*>(group_rows<NR, OV>(P, ys, g)) + c;
    for (int r = r0 + lane; r < P.l; r += 32) put_tagged<real>(dst + (int64_t)r * W, tag, src[4 * (int64_t)r]);
  }
}

// All threads of step j, after the barrier that follows decide_pivot: the
// pivot column x that its owner published (tagged words), its norm nu, and
// the step's reflector (beta, tau, scale).  Float32: xv receives the
// Householder vector itself, v(r) = 0 above row j (row j - 1 is cleared
// here, the rows above it in earlier steps), v(j) = 1, v(r) = scale x(r)
// below; every thread reads x(j) and forms the reflector, so one barrier ends
// the fetch.  Float64 (divisions and products at a 64th of the float32 rate):
// xv receives x itself (rows j..l-1), thread 0 forms the reflector and a
// second barrier shares it; the update folds scale into its sums.  False
// (st.stop = 2, the abort flag raised) if a word never became fresh.
template <typename real>
__device__ __forceinline__ bool fetch_v(const CpqrParams<real>& P, int j, int owner, real nu,
                                        real* xv, StepState<real>& st, real* beta, real* tau,
                                        real* scale) {
  constexpr int W = Words<real>::W;
  const int tid = threadIdx.x, l = P.l;
  const unsigned long long* src = slot_of(P, j & 1, owner);
  const unsigned tag = tag_of(P.gen, j + 1);
  bool ok = true;
  if constexpr (sizeof(real) == 4) {
    real alpha = real(0);
    if (!get_tagged<real>(src + (int64_t)j * W, tag, &alpha, P.abort_flag, P.spin)) ok = false;
    reflector(alpha, nu, beta, tau, scale);
    for (int r = j + tid; r < l; r += kThreads) {
      real x = alpha;
      if (r > j && !get_tagged<real>(src + (int64_t)r * W, tag, &x, P.abort_flag, P.spin)) {
        ok = false;
        x = real(0);
      }
      xv[r] = r == j ? real(1) : *scale * x;
    }
    if (j > 0 && tid == kThreads - 1) xv[j - 1] = real(0);
    if (!ok) st.stale = 1;
    cta_sync();
  } else {
    for (int r = j + tid; r < l; r += kThreads) {
      real x;
      if (!get_tagged<real>(src + (int64_t)r * W, tag, &x, P.abort_flag, P.spin)) {
        ok = false;
        x = real(0);
      }
      xv[r] = x;
    }
    if (!ok) st.stale = 1;
    cta_sync();
    if (tid == 0) reflector(xv[j], nu, &st.beta, &st.tau, &st.scale);
    cta_sync();
    *beta = st.beta;
    *tau = st.tau;
    *scale = st.scale;
  }
  if (st.stale) {
    if (tid == 0) {
      atomicExch(P.abort_flag, 1);
      set_flag(&P.status->flags, FLAG_TIMEOUT);
    }
    st.stop = 2;
    return false;
  }
  return true;
}

// H applied to a register-resident group (rows lane + 32 u), v = xv (zero
// above row j and past l, so neither pass needs a row mask but the norms';
// every row block is processed: skipping the blocks above j, a branch per
// block, measured slower).  act: the group's unselected columns other than
// the pivot; pc: the pivot's column in the group, or -1.
template <int RPL, typename real>
__device__ __forceinline__ void update_reg_group(Quad<real> (&y)[RPL], const real* xv, int j,
                                                 real tau, real beta, unsigned act, int pc,
                                                 int lane, int g, LaneBest<real>& best) {
  real d0 = real(0), d1 = real(0), d2 = real(0), d3 = real(0);
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const real v = xv[lane + 32 * u];
    d0 += v * y[u].x;
    d1 += v * y[u].y;
    d2 += v * y[u].z;
    d3 += v * y[u].w;
  }
  const int cs = (lane >> 3) & 3;
  const bool on = (act >> cs) & 1u;
  const real dg = reduce4(d0, d1, d2, d3, lane);  // every lane: full-warp shuffles
  const real w = on ? tau * dg : real(0);
  const real w0 = __shfl_sync(0xffffffffu, w, 0), w1 = __shfl_sync(0xffffffffu, w, 8);
  const real w2 = __shfl_sync(0xffffffffu, w, 16), w3 = __shfl_sync(0xffffffffu, w, 24);
  real q0 = real(0), q1 = real(0), q2 = real(0), q3 = real(0);
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const int r = lane + 32 * u;
    const real v = xv[r];
    y[u].x -= w0 * v;
    y[u].y -= w1 * v;
    y[u].z -= w2 * v;
    y[u].w -= w3 * v;
    if (r > j) {
      q0 += y[u].x * y[u].x;
      q1 += y[u].y * y[u].y;
      q2 += y[u].z * y[u].z;
      q3 += y[u].w * y[u].w;
    }
  }
  if (pc >= 0) {
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      if (32 * u + 31 < j) continue;
      const int r = lane + 32 * u;
      if (r >= j) set_comp(y[u], pc, r == j ? beta : real(0));
    }
  }
  const real qg = reduce4(q0, q1, q2, q3, lane);
  if (on) best.add(qg, 4 * g + cs);
}

// H applied to a group in shared or global memory (yg: its rows); rows
// above j are not touched.  Float32, v = xv: w = tau v^T y over rows
// j..l-1, y -= w v.  Float64, x = xv: w = tau (y(j) + scale x^T y over rows
// j+1..l-1), y(j) -= w, y -= (w scale) x below.  Lane 0 updates row j, whose
// new values do not enter the residual norms.
template <int UNROLL, typename real>
__device__ __forceinline__ void update_mem_group(Quad<real>* yg, const real* xv, int l, int j,
                                                 real tau, real beta, real scale, unsigned act,
                                                 int pc, int lane, int g, LaneBest<real>& best) {
  constexpr bool RAW = sizeof(real) == 8;
  real d0 = real(0), d1 = real(0), d2 = real(0), d3 = real(0);
#pragma unroll UNROLL
  for (int r = j + (RAW ? 1 : 0) + lane; r < l; r += 32) {
    const real v = xv[r];
    const Quad<real> t = ldq(yg + r);
    d0 += v * t.x;
    d1 += v * t.y;
    d2 += v * t.z;
    d3 += v * t.w;
  }
  const int cs = (lane >> 3) & 3;
  const bool on = (act >> cs) & 1u;
  Quad<real> yj;
  if (RAW) yj = ldq(yg + j);  // every lane, before the shuffles below
  const real dg = reduce4(d0, d1, d2, d3, lane);
  const real w = on ? (RAW ? tau * (comp(yj, cs) + scale * dg) : tau * dg) : real(0);
  const real w0 = __shfl_sync(0xffffffffu, w, 0), w1 = __shfl_sync(0xffffffffu, w, 8);
  const real w2 = __shfl_sync(0xffffffffu, w, 16), w3 = __shfl_sync(0xffffffffu, w, 24);
  // every lane's reads of row j are done (they fed the w it shuffled)
  if (lane == 0) {
    Quad<real> t = ldq(yg + j);
    t.x -= w0;
    t.y -= w1;
    t.z -= w2;
    t.w -= w3;
    stq(yg + j, t);
  }
  const real s0 = RAW ? w0 * scale : w0, s1 = RAW ? w1 * scale : w1;
  const real s2 = RAW ? w2 * scale : w2, s3 = RAW ? w3 * scale : w3;
  real q0 = real(0), q1 = real(0), q2 = real(0), q3 = real(0);
#pragma unroll UNROLL
  for (int r = j + 1 + lane; r < l; r += 32) {
    const real v = xv[r];
    Quad<real> t = ldq(yg + r);
    t.x -= s0 * v;
    t.y -= s1 * v;
    t.z -= s2 * v;
    t.w -= s3 * v;
    q0 += t.x * t.x;
    q1 += t.y * t.y;
    q2 += t.z * t.z;
    q3 += t.w * t.w;
    stq(yg + r, t);
  }
  if (pc >= 0) {
    // the pivot column: beta at row j, zeros below (its w is zero, so the
    // passes above left it as it was); each lane rewrites rows it stored
    real* col = reinterpret_cast<real*>(yg) + pc;
    if (lane == 0) col[4 * (int64_t)j] = beta;
    for (int r = j + 1 + lane; r < l; r += 32) col[4 * (int64_t)r] = real(0);
  }
  const real qg = reduce4(q0, q1, q2, q3, lane);
  if (on) best.add(qg, 4 * g + cs);
}

// For short columns (the 7-row register groups) a group's fixed costs -- two
// shuffle reductions, the w broadcast, the best-column bookkeeping -- outweigh
// its row work, so the update is split in two halves and a warp runs its
// memory groups two at a time (their reductions overlap):
//   dots:  lane-partial sums of v^T y for the four columns;
//   apply: y -= w v with the w of the four columns, lane-partial squared
//          norms of rows j+1..l-1, and the pivot column retired (beta at row
//          j, zeros below; its w is zero, so the update leaves it as it was).
// Register groups hold rows lane + 32 u; v = xv is zero above row j and past
// l, so they need no row mask but the norms' (Section 2.2's residual norms
// over rows j+1..l-1).  Groups in shared or global memory (yg: their rows)
// are not touched above row j.  Float32: xv holds v, w = tau v^T y over rows
// j..l-1.  Float64: xv holds the pivot column x, w = tau (y(j) + scale x^T y
// over rows j+1..l-1), y(j) -= w and y -= (w scale) x below.

template <int RPL, typename real>
__device__ __forceinline__ void reg_dots(const Quad<real> (&y)[RPL], const real* xv, int lane,
                                         real (&d)[4]) {
  d[0] = d[1] = d[2] = d[3] = real(0);
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const real v = xv[lane + 32 * u];
    d[0] += v * y[u].x;
    d[1] += v * y[u].y;
    d[2] += v * y[u].z;
    d[3] += v * y[u].w;
  }
}

template <int RPL, typename real>
__device__ __forceinline__ void reg_apply(Quad<real> (&y)[RPL], const real* xv, int j,
                                          const real (&w)[4], int pc, real beta, int lane,
                                          real (&q)[4]) {
  q[0] = q[1] = q[2] = q[3] = real(0);
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const int r = lane + 32 * u;
    const real v = xv[r];
    y[u].x -= w[0] * v;
    y[u].y -= w[1] * v;
    y[u].z -= w[2] * v;
    y[u].w -= w[3] * v;
    if (r > j) {
      q[0] += y[u].x * y[u].x;
      q[1] += y[u].y * y[u].y;
      q[2] += y[u].z * y[u].z;
      q[3] += y[u].w * y[u].w;
    }
  }
  if (pc >= 0) {
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      if (32 * u + 31 < j) continue;
      const int r = lane + 32 * u;
      if (r >= j) set_comp(y[u], pc, r == j ? beta : real(0));
    }
  }
}

template <int UNROLL, typename real>
__device__ __forceinline__ void mem_dots(const Quad<real>* yg, const real* xv, int l, int j,
                                         int lane, real (&d)[4]) {
  constexpr bool RAW = sizeof(real) == 8;
  d[0] = d[1] = d[2] = d[3] = real(0);
#pragma unroll UNROLL
  for (int r = j + (RAW ? 1 : 0) + lane; r < l; r += 32) {
    const real v = xv[r];
    const Quad<real> t = ldq(yg + r);
    d[0] += v * t.x;
    d[1] += v * t.y;
    d[2] += v * t.z;
    d[3] += v * t.w;
  }
}

// w of the lane's column cs from its reduced dot product dg (zero unless on)
template <typename real>
__device__ __forceinline__ real mem_w(const Quad<real>* yg, int j, real dg, real tau, real scale,
                                      bool on, int cs) {
  if constexpr (sizeof(real) == 8) return on ? tau * (comp(ldq(yg + j), cs) + scale * dg) : real(0);
  return on ? tau * dg : real(0);
}

template <int UNROLL, typename real>
__device__ __forceinline__ void mem_apply(Quad<real>* yg, const real* xv, int l, int j,
                                          const real (&w)[4], real scale, int pc, real beta,
                                          int lane, real (&q)[4]) {
  constexpr bool RAW = sizeof(real) == 8;
  // every lane's reads of row j are done (they fed the w it shuffled)
  if (lane == 0) {
    Quad<real> t = ldq(yg + j);
    t.x -= w[0];
    t.y -= w[1];
    t.z -= w[2];
    t.w -= w[3];
    stq(yg + j, t);
  }
  const real s0 = RAW ? w[0] * scale : w[0], s1 = RAW ? w[1] * scale : w[1];
  const real s2 = RAW ? w[2] * scale : w[2], s3 = RAW ? w[3] * scale : w[3];
  q[0] = q[1] = q[2] = q[3] = real(0);
#pragma unroll UNROLL
  for (int r = j + 1 + lane; r < l; r += 32) {
    const real v = xv[r];
    Quad<real> t = ldq(yg + r);
    t.x -= s0 * v;
    t.y -= s1 * v;
    t.z -= s2 * v;
    t.w -= s3 * v;
    q[0] += t.x * t.x;
    q[1] += t.y * t.y;
    q[2] += t.z * t.z;
    q[3] += t.w * t.w;
    stq(yg + r, t);
  }
  if (pc >= 0) {
    // each lane rewrites rows it stored
    real* col = reinterpret_cast<real*>(yg) + pc;
    if (lane == 0) col[4 * (int64_t)j] = beta;
    for (int r = j + 1 + lane; r < l; r += 32) col[4 * (int64_t)r] = real(0);
  }
}

// The four columns' values of lane 8 c (c = 0..3) to every lane.
template <typename real>
__device__ __forceinline__ void bcast4(real x, real (&w)[4]) {
  w[0] = __shfl_sync(0xffffffffu, x, 0);
  w[1] = __shfl_sync(0xffffffffu, x, 8);
  w[2] = __shfl_sync(0xffffffffu, x, 16);
  w[3] = __shfl_sync(0xffffffffu, x, 24);
}

// Squared norms of the columns of a group in memory, all rows.
template <typename real>
__device__ __forceinline__ real mem_group_norms(const Quad<real>* yg, int l, int lane) {
  real q0 = real(0), q1 = real(0), q2 = real(0), q3 = real(0);
  for (int r = lane; r < l; r += 32) {
    const Quad<real> t = ldq(yg + r);
    q0 += t.x * t.x;
    q1 += t.y * t.y;
    q2 += t.z * t.z;
    q3 += t.w * t.w;
  }
  return reduce4(q0, q1, q2, q3, lane);
}

// The steps of the factorization as one warp runs them (every warp calls it
// once; all take the same CTA barriers, as cta_sync: warp 0 reaches them
// from its own copy of this function).  LEAD: warp 0, which gathers the
// records and holds no register group, so its registers never carry both
// the records in flight and a register group.  Returns the steps taken.
template <typename real, int RPL, bool OV, bool LEAD>
__device__ __forceinline__ int cpqr_steps(const CpqrParams<real>& P, Quad<real>* ys, real* xv,
                                          int* active, StepState<real>& st, WarpBest<real>& wb,
                                          int c0, int ncl, int ng, int* k_eff_out) {
  constexpr int NR = RPL > 0 ? kWarps - 1 : 0;  // register groups of a CTA
  constexpr bool REGS = RPL > 0 && !LEAD;        // this warp holds one
  constexpr int RR = REGS ? RPL : 1;
  constexpr int UN = 4;  // rows in flight per lane in the memory groups' loops
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = P.l;
  const int g0 = warp - 1;  // the register group, for warps 1..15
  const int cs = (lane >> 3) & 3;
  Quad<real> yr[RR];
#pragma unroll
  for (int u = 0; u < RR; ++u) yr[u] = Quad<real>{real(0), real(0), real(0), real(0)};
  const bool has_reg = REGS && g0 >= 0 && g0 < ng;
  if (has_reg) {
    const int lc = 4 * g0;
#pragma unroll
    for (int u = 0; u < RR; ++u) {
      const int r = lane + 32 * u;
      if (r < l) {
        const real* row = P.Y + (int64_t)r * P.ldy + c0 + lc;
        yr[u].x = lc < ncl ? row[0] : real(0);
        yr[u].y = lc + 1 < ncl ? row[1] : real(0);
        yr[u].z = lc + 2 < ncl ? row[2] : real(0);
        yr[u].w = lc + 3 < ncl ? row[3] : real(0);
      }
    }
  }
  cta_sync();  // groups in memory loaded, active flags set
  LaneBest<real> best;
  best.reset();
  if (has_reg) {
    real q0 = real(0), q1 = real(0), q2 = real(0), q3 = real(0);
#pragma unroll
    for (int u = 0; u < RR; ++u) {
      q0 += yr[u].x * yr[u].x;
      q1 += yr[u].y * yr[u].y;
      q2 += yr[u].z * yr[u].z;
      q3 += yr[u].w * yr[u].w;
    }
    const real qg = reduce4(q0, q1, q2, q3, lane);
    if ((act_of(active, g0) >> cs) & 1u) best.add(qg, 4 * g0 + cs);
  }
  for (int g = first_mem_group<NR>(warp); g < ng; g = next_mem_group<NR>(g)) {
    const real qg = mem_group_norms(group_rows<NR, OV>(P, ys, g), l, lane);
    if ((act_of(active, g) >> cs) & 1u) best.add(qg, 4 * g + cs);
  }
  post_best(best, lane, warp, wb);
  cta_sync();
  publish<RR, REGS, NR, OV>(P, ys, wb, yr, c0, 0, 0, 1u, lane, warp);

  real normY = real(-1), nu_first = real(0);
  int k_eff = -1;
  int j = 0;
  for (;; ++j) {
    if (LEAD) decide_pivot(P, j, normY, st);
    cta_sync();
    if (st.stop) break;
    const int owner = st.owner, pcol = st.col;
    const real nu = st.nu;
    note_rank(P, j, nu, nu_first, k_eff);
    real beta, tau, scale;
    if (!fetch_v(P, j, owner, nu, xv, st, &beta, &tau, &scale)) break;
    const int pl = pcol - c0;                             // local pivot column
    const int pg = (pl >= 0 && pl < ncl) ? pl >> 2 : -1;  // its group, if here
    best.reset();
    if constexpr (RPL != kGroupRegRowsShort) {
      if (has_reg) {
        const int pc = pg == g0 ? pl & 3 : -1;
        const unsigned act = act_of(active, g0) & ~(pc >= 0 ? 1u << pc : 0u);
        if (act || pc >= 0)
          update_reg_group<RR>(yr, xv, j, tau, beta, act, pc, lane, g0, best);
      }
      for (int g = first_mem_group<NR>(warp); g < ng; g = next_mem_group<NR>(g)) {
        const int pc = pg == g ? pl & 3 : -1;
        const unsigned act = act_of(active, g) & ~(pc >= 0 ? 1u << pc : 0u);
        if (!act && pc < 0) continue;
        const int s = g - NR;
        if (!OV || s < P.ncs)
          update_mem_group<UN>(ys + (int64_t)s * l, xv, l, j, tau, beta, scale, act, pc, lane, g,
                               best);
        else
          update_mem_group<UN>(group_rows<NR, true>(P, ys, g), xv, l, j, tau, beta, scale, act, pc,
                               lane, g, best);
      }
    } else {
      // the register group, then the memory groups two by two: each pair's
      // dots, their reductions, the w's, the updates, the norms' reductions
      // (retired columns get w = 0)
      int g = first_mem_group<NR>(warp);
      auto mem_rows = [&](int gg) -> Quad<real>* {
        const int s = gg - NR;
        return (!OV || s < P.ncs) ? ys + (int64_t)s * l : group_rows<NR, true>(P, ys, gg);
      };
      auto pivot_in = [&](int gg) { return pg == gg ? pl & 3 : -1; };
      auto act_in = [&](int gg, int pc) {
        return act_of(active, gg) & ~(pc >= 0 ? 1u << pc : 0u);
      };
      if (has_reg) {
        const int pcA = pivot_in(g0);
        const bool onA = (act_in(g0, pcA) >> cs) & 1u;
        real dA[4], wA[4];
        reg_dots<RR>(yr, xv, lane, dA);
        const real rA = reduce4(dA[0], dA[1], dA[2], dA[3], lane);
        bcast4(onA ? tau * rA : real(0), wA);
        reg_apply<RR>(yr, xv, j, wA, pcA, beta, lane, dA);
        const real qA = reduce4(dA[0], dA[1], dA[2], dA[3], lane);
        if (onA) best.add(qA, 4 * g0 + cs);
      }
      while (g < ng) {
        const int g2 = next_mem_group<NR>(g);
        const bool B = g2 < ng;
        Quad<real>* yA = mem_rows(g);
        Quad<real>* yB = B ? mem_rows(g2) : yA;
        const int pcA = pivot_in(g), pcB = B ? pivot_in(g2) : -1;
        const bool onA = (act_in(g, pcA) >> cs) & 1u;
        const bool onB = B && ((act_in(g2, pcB) >> cs) & 1u);
        real dA[4], dB[4];
        mem_dots<UN>(yA, xv, l, j, lane, dA);
        if (B) mem_dots<UN>(yB, xv, l, j, lane, dB);
        const real rA = reduce4(dA[0], dA[1], dA[2], dA[3], lane);
        const real rB = B ? reduce4(dB[0], dB[1], dB[2], dB[3], lane) : real(0);
        real wA[4], wB[4];
        bcast4(mem_w(yA, j, rA, tau, scale, onA, cs), wA);
        if (B) bcast4(mem_w(yB, j, rB, tau, scale, onB, cs), wB);
        mem_apply<UN>(yA, xv, l, j, wA, scale, pcA, beta, lane, dA);
        if (B) mem_apply<UN>(yB, xv, l, j, wB, scale, pcB, beta, lane, dB);
        const real qA = reduce4(dA[0], dA[1], dA[2], dA[3], lane);
        const real qB = B ? reduce4(dB[0], dB[1], dB[2], dB[3], lane) : real(0);
        if (onA) best.add(qA, 4 * g + cs);
        if (onB) best.add(qB, 4 * g2 + cs);
        g = B ? next_mem_group<NR>(g2) : g2;
      }
    }
    if (pg >= 0 && group_owner<NR>(pg) == warp && lane == 0) {
      active[pl] = 0;
      P.J[j] = pcol;
    }
    post_best(best, lane, warp, wb);
    cta_sync();
    publish<RR, REGS, NR, OV>(P, ys, wb, yr, c0, j + 1, (j + 1) & 1, (unsigned)(j + 2), lane, warp);
  }
  *k_eff_out = k_eff;
  // rows 0..j-1 of S from the register group
  if (has_reg && st.stop != 2) {
#pragma unroll
    for (int u = 0; u < RR; ++u) {
      const int r = lane + 32 * u;
      if (r >= j) continue;
      real* row = P.S + (int64_t)r * P.lds + c0 + 4 * g0;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (4 * g0 + c < ncl) row[c] = comp(yr[u], c);
    }
  }
  return j;
}

// RPL > 0: the first group of warps 1..15 is register-resident (RPL rows
// per lane).  OV: some groups live in the global overflow area.
template <typename real, int RPL, bool OV>
__global__ void __launch_bounds__(kThreads, 1) cpqr_kernel(CpqrParams<real> P) {
  constexpr int NR = RPL > 0 ? kWarps - 1 : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int b = blockIdx.x;
  const int nc = P.nc, l = P.l;
  Quad<real>* ys = reinterpret_cast<Quad<real>*>(smem_raw);  // P.ncs groups of l rows
  real* xv = reinterpret_cast<real*>(ys + (int64_t)P.ncs * l);  // pivot column of the step
  int* active = reinterpret_cast<int*>(xv + P.ldl);             // nc flags
  // (P.ldl: l rounded up to 4, at least the rows of the register groups)

  __shared__ StepState<real> st;
  __shared__ WarpBest<real> wb;

  const int c0 = b * nc;
  const int ncl = max(0, min(nc, P.n - c0));
  const int ng = (ncl + 3) >> 2;  // groups holding this CTA's columns

  for (int lc = tid; lc < nc; lc += kThreads) active[lc] = lc < ncl ? 1 : 0;
  for (int r = tid; r < P.ldl; r += kThreads) xv[r] = real(0);
  // groups in memory, read along the rows of Y; the columns past ncl of the
  // last group are zero
  const int cm0 = min(4 * ng, 4 * NR), ncm = 4 * ng - cm0;
  for (int64_t e = tid; e < (int64_t)l * ncm; e += kThreads) {
    const int r = (int)(e / ncm), lc = cm0 + (int)(e % ncm);
    const real yv = lc < ncl ? P.Y[(int64_t)r * P.ldy + c0 + lc] : real(0);
    reinterpret_cast<real*>(group_rows<NR, OV>(P, ys, lc >> 2) + r)[lc & 3] = yv;
  }
  int k_eff = -1;
  const int k_done = warp == 0
                         ? cpqr_steps<real, RPL, OV, true>(P, ys, xv, active, st, wb, c0, ncl, ng, &k_eff)
                         : cpqr_steps<real, RPL, OV, false>(P, ys, xv, active, st, wb, c0, ncl, ng, &k_eff);
  if (st.stop == 2) return;  // timed out: leave without further waits
  // S rows 0..k_done-1 of the groups in memory, in original column order
  for (int64_t e = tid; e < (int64_t)k_done * ncm; e += kThreads) {
    const int i = (int)(e / ncm), lc = cm0 + (int)(e % ncm);
    if (lc < ncl)
      P.S[(int64_t)i * P.lds + c0 + lc] =
          reinterpret_cast<const real*>(group_rows<NR, OV>(P, ys, lc >> 2) + i)[lc & 3];
  }
  finish_order(P, active, ncl, c0, k_done, k_eff, st);
}

// Shape of one factorization: grid, columns per CTA (a multiple of four),
// which kernel, and for the grouped kernel its register rows, groups in
// shared memory and overflow groups per CTA.
struct Layout {
  int G = 1, nc = 4, warps = kWarps;
  bool reg = false;  // the register-resident kernel (cpqr_reg.cu)
  int rpl = 0;       // grouped kernel: rows per lane of the register groups
  int ncs = 0;       // grouped kernel: groups in shared memory
  int ngo = 0;       // grouped kernel: overflow groups per CTA
  int ldl = 1;
  size_t smem = 0;
};

// rows of the step's Householder vector in shared memory: l rounded up to a
// multiple of 4, at least the rows of the register groups
inline int64_t grouped_v_rows(int64_t l, int rpl) {
  return std::max<int64_t>((l + 3) & ~int64_t(3), 32 * (int64_t)rpl);
}

template <typename real>
size_t grouped_smem_bytes(int ncs, int nc, int64_t l, int rpl) {
  return (size_t)ncs * l * 4 * sizeof(real) + (size_t)grouped_v_rows(l, rpl) * sizeof(real) +
         (size_t)nc * sizeof(int) + 64;
}

// Grid, columns per CTA and kernel of an l x n factorization.
//
// One decomposition at a time (the handle's concurrency 1): one CTA per SM,
// the lowest latency per factorization.  With two to seven in flight: the
// fewest CTAs whose registers hold the matrix (eight columns per warp of the
// register-resident kernel).  The pivot exchange gets cheaper with fewer
// CTAs (records of 38-64 CTAs meet in about 2.4K cycles on GB300, of 152 in
// about twice that), the update gets longer, and the SMs left free run the
// other decompositions: the factorization takes about 1.2x as long on a
// third of the SMs.  With eight or more in flight (float32): the grouped
// kernel on the fewest CTAs whose registers and shared memory hold the
// matrix (about 330 columns of 210 rows per CTA): about twice as long again
// on a third of those SMs, which pays once enough decompositions share the
// GPU (8000 x 6000, k = 200: 766/s with eight in flight against 653/s for
// the register kernel; 528/s against 617/s with four).  Cooperative grids
// are gang-scheduled, so grids of concurrent factorizations queue whole.
// In the environment, for comparisons: CURID_CPQR_CTAS = "all" (one per SM),
// "fewest" or a number of CTAs; CURID_CPQR_KERNEL = "grouped" or "reg".
// (Eight-warp CTAs, two per SM, so that two concurrent factorizations share
// SMs, measured slower: 549/s against 613/s with four in flight.)
template <typename real>
curid_status cpqr_layout(const Ctx& ctx, int64_t l, int64_t n, Layout* L) {
  if (l <= 0 || n <= 0) return CURID_INVALID_ARG;
  if (l > (1 << 24) || n > INT32_MAX / 2) return CURID_UNSUPPORTED;
  const int gmax = std::min(ctx.num_sms, 32 * kMaxSlotsPerLane);
  int G = (int)std::min<int64_t>(gmax, n);
  const char* env = std::getenv("CURID_CPQR_CTAS");
  bool fewest = ctx.concurrency > 1;
  if (env && std::strcmp(env, "all") == 0) fewest = false;
  if (env && std::strcmp(env, "fewest") == 0) fewest = true;
  const char* kenv = std::getenv("CURID_CPQR_KERNEL");
  const int rpl = group_reg_rows<real>(l);
  // eight or more in flight (float32): the grouped kernel on the fewest CTAs
  bool force_grouped = fewest && ctx.concurrency >= 8 && rpl > 0;
  if (kenv && std::strcmp(kenv, "grouped") == 0) force_grouped = true;
  if (kenv && std::strcmp(kenv, "reg") == 0) force_grouped = false;
  const int forced_g = env ? std::atoi(env) : 0;  // a number: that many CTAs (comparisons)
  if (forced_g > 0) {
    G = (int)std::min<int64_t>(std::min(forced_g, gmax), n);
  } else if (fewest && force_grouped) {
    // fewest CTAs whose registers and shared memory hold the matrix
    const int64_t nr = rpl > 0 ? kWarps - 1 : 0;
    for (int g = 1; g <= gmax; ++g) {
      const int64_t ncg = (((n + g - 1) / g) + 3) & ~int64_t(3);
      const size_t fixed = grouped_smem_bytes<real>(0, (int)ncg, l, rpl) + 1024;
      if (fixed > ctx.smem_optin) continue;
      const int64_t cap = nr + (int64_t)((ctx.smem_optin - fixed) / ((size_t)l * 4 * sizeof(real)));
      if (ncg / 4 <= cap) {
        G = g;
        break;
      }
    }
  } else if (fewest) {
    const int64_t rc = cpqr_reg_cols<real>((int)l, kWarps);
    if (rc > 0 && (n + rc - 1) / rc <= gmax) G = (int)((n + rc - 1) / rc);
  }
  int nc = (int)((n + G - 1) / G);
  nc = (nc + 3) & ~3;
  G = (int)((n + nc - 1) / nc);
  L->G = G;
  L->nc = nc;
  L->warps = kWarps;
  L->reg = !force_grouped && cpqr_reg_fits<real>(ctx, (int)l, nc, kWarps);
  if (L->reg) {
    L->ldl = (int)(l | 1);
    L->rpl = L->ncs = L->ngo = 0;
    L->smem = 0;  // cpqr_reg_launch sizes its own
    return CURID_OK;
  }
  L->rpl = rpl;
  const int nr = L->rpl > 0 ? kWarps - 1 : 0;
  const int rest = std::max(0, nc / 4 - nr);
  // the kernel's static shared variables share the per-block limit
  const size_t fixed = grouped_smem_bytes<real>(0, nc, l, L->rpl) + 1024;
  if (fixed > ctx.smem_optin) return CURID_UNSUPPORTED;
  L->ncs = (int)std::min<size_t>(rest, (ctx.smem_optin - fixed) / ((size_t)l * 4 * sizeof(real)));
  L->ngo = rest - L->ncs;
  L->ldl = (int)grouped_v_rows(l, L->rpl);
  L->smem = grouped_smem_bytes<real>(L->ncs, nc, l, L->rpl);
  return CURID_OK;
}

template <typename real>
void (*grouped_kernel(const Layout& L))(CpqrParams<real>) {
  if constexpr (sizeof(real) == 4) {
    if (L.rpl == kGroupRegRows)
      return L.ngo > 0 ? cpqr_kernel<real, kGroupRegRows, true> : cpqr_kernel<real, kGroupRegRows, false>;
    if (L.rpl == kGroupRegRowsShort)
      return L.ngo > 0 ? cpqr_kernel<real, kGroupRegRowsShort, true>
                       : cpqr_kernel<real, kGroupRegRowsShort, false>;
  }
  if (L.rpl != 0) return nullptr;
  return L.ngo > 0 ? cpqr_kernel<real, 0, true> : cpqr_kernel<real, 0, false>;
}

}  // namespace

template <typename real>
curid_status cpqr_plan(const Ctx& ctx, int64_t l, int64_t n, int* grid, size_t* smem) {
  Layout L;
  CURID_TRY(cpqr_layout<real>(ctx, l, n, &L));
  *grid = L.G;
  *smem = L.smem;
  return CURID_OK;
}

template <typename real>
void cpqr_carve(Carver& cv, const Ctx& ctx, int64_t l, int64_t n, CpqrScratch* s) {
  Layout L;
  if (cpqr_layout<real>(ctx, l, n, &L) != CURID_OK) L = Layout();
  s->grid = L.G;
  s->slots = cv.take<Rec>(2 * (size_t)L.G);
  s->slot_data = cv.take<unsigned long long>(2 * (size_t)L.G * slot_words<real>(l));
  s->counts = cv.take<int>(L.G);
  s->abort_flag = cv.take<int>(1);
  s->overflow = L.ngo > 0 ? cv.take<real>((size_t)L.G * L.ngo * (size_t)l * 4) : nullptr;
}

template <typename real>
curid_status cpqr_run(const Ctx& ctx, const real* Y, int64_t l, int64_t n, int64_t ldy, int k_max,
                      double tol, int32_t* J, real* S, int64_t lds, const CpqrScratch& s,
                      int which) {
  Layout L;
  CURID_TRY(cpqr_layout<real>(ctx, l, n, &L));
  if (L.G != s.grid || (L.ngo > 0 && !s.overflow)) return CURID_INVALID_ARG;
  CpqrParams<real> P;
  P.Y = Y;
  P.ldy = ldy;
  P.l = (int)l;
  P.n = (int)n;
  P.k_max = k_max;
  P.nc = L.nc;
  P.ncs = L.ncs;
  P.gys = static_cast<real*>(s.overflow);
  P.ldl = L.ldl;
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
  P.warps = L.warps;
  CURID_CUDA(cudaMemsetAsync(s.slots, 0, 2 * (size_t)L.G * sizeof(Rec), ctx.stream));
  CURID_CUDA(cudaMemsetAsync(s.abort_flag, 0, sizeof(int), ctx.stream));
  if (L.reg) return cpqr_reg_launch<real>(ctx, P, L.G);
  auto fn = grouped_kernel<real>(L);
  if (!fn) return CURID_UNSUPPORTED;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
  void* args[] = {&P};
  CURID_CUDA(cudaLaunchCooperativeKernel((void*)fn, dim3(L.G), dim3(kThreads), args, L.smem,
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
