// Grid-wide pivot exchange shared by the persistent CPQR kernels (the
// shared-memory slab kernel in cpqr.cu and the register-resident one in
// cpqr_reg.cu): per-step records, tagged candidate columns, the pivot
// decision of a step, the read of the pivot column and the closing exchange
// that orders the unselected columns (Section 2.2, Eq. (2.4)-(2.5)).
#pragma once

#include "kernels.cuh"

namespace curid {
namespace cpqr_x {

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
  int ncs;                       // grouped kernel: column groups in shared memory
  real* gys;                     // grouped kernel: [G][overflow groups][l][4] the rest
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
  long long spin;                // bound of every inter-block wait, SM clock cycles
  int warps;                     // warps per CTA of the register-resident kernel
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

// Words of one candidate slot: rows 0..l-1 of the column.
template <typename real>
__host__ __device__ constexpr int64_t slot_words(int64_t l) {
  return l * Words<real>::W;
}

// Slot of CTA `cta` in exchange buffer bf.
template <typename real>
__device__ __forceinline__ unsigned long long* slot_of(const CpqrParams<real>& P, int bf, int cta) {
  return P.slot_data + ((int64_t)bf * gridDim.x + cta) * slot_words<real>(P.l);
}

// CTA barrier that may be reached from different instructions by different
// warps (PTX barrier.sync without .aligned): the grouped kernel runs warp 0
// and the other warps through two copies of the step loop.  Same memory
// ordering as __syncthreads().
__device__ __forceinline__ void cta_sync() { asm volatile("barrier.sync 0;" ::: "memory"); }

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
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
    st_gpu_u64(dst, pack(tag, (unsigned)(b >> 32)));
    st_gpu_u64(dst + 1, pack(tag, (unsigned)(b & 0xffffffffull)));
  } else {
    st_gpu_u64(dst, pack(tag, __float_as_uint((float)v)));
  }
}

// Bounded read of one tagged element; false if it never became fresh.
template <typename real>
__device__ __forceinline__ bool get_tagged(const unsigned long long* src, unsigned tag, real* v,
                                           const int* abort_flag, long long spin) {
  const long long t0 = clock64();
  while (true) {
    if (sizeof(real) == 8) {
      const unsigned long long a = ld_gpu_u64(src), b = ld_gpu_u64(src + 1);
      if ((unsigned)(a >> 32) == tag && (unsigned)(b >> 32) == tag) {
        *v = (real)__longlong_as_double((long long)(((a & 0xffffffffull) << 32) |
                                                     (b & 0xffffffffull)));
        return true;
      }
    } else {
      const unsigned long long a = ld_gpu_u64(src);
      if ((unsigned)(a >> 32) == tag) {
        *v = (real)__uint_as_float((unsigned)(a & 0xffffffffull));
        return true;
      }
    }
    if (ld_gpu_i32(abort_flag) || clock64() - t0 > spin) return false;
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
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(&r->w[0]), "l"(a), "l"(b)
               : "memory");
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(&r->w[2]), "l"(c), "l"(d)
               : "memory");
}

__device__ __forceinline__ void ld_rec(const Rec* r, unsigned long long* w) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];"
               : "=l"(w[0]), "=l"(w[1])
               : "l"(&r->w[0]));
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];"
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
        asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];"
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
    // the clock every round (no memory access), the abort flag every 16th
    // (a load that would otherwise lengthen every polling round)
    if (clock64() - t0 > P.spin) {
      atomicExch(P.abort_flag, 1);
      ok = false;
      break;
    }
    if ((round & 15) == 15 && ld_gpu_i32(P.abort_flag)) { ok = false; break; }
  }
  ok = __all_sync(0xffffffffu, ok);
  return ok;
}


// Per-step decision shared by the threads of a CTA.
template <typename real>
struct StepState {
  int stop;    // 0: go on, 1: done, 2: timed out / aborted
  int owner;   // CTA that published the pivot column
  int col;     // pivot column (global index)
  int prefix;  // closing exchange: unselected columns of lower CTAs
  int stale;   // a tagged word of the pivot column never became fresh
  real nu;     // pivot norm
  real beta, tau, scale;  // the step's reflector (float64: formed once per CTA)
};

// Warp 0 of step j: gather the G records of the step, pick the global pivot
// (largest residual norm, smallest column on ties) and decide whether to
// stop (k_max reached, no column left, a non-finite norm, the tolerance
// ||Y - Q_j Q_j^T Y||_F <= tol ||Y||_F met, or a timeout).  normY is kept by
// lane 0 between steps.  Results in st (read after a CTA barrier).
template <typename real>
__device__ __forceinline__ void decide_pivot(const CpqrParams<real>& P, int j, real& normY,
                                             StepState<real>& st) {
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x, b = blockIdx.x;
  unsigned long long w[kMaxSlotsPerLane][4];
  const bool ok = gather_records(P, j & 1, tag_of(P.gen, j + 1), w);
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
    st.stop = stop;
    // every read of the previous step's stale flag came before the barrier
    // that ended that step's update
    st.stale = 0;
    st.owner = bo;
    st.col = (int)bc;
    st.nu = bn;
  }
}

// All threads of step j, after the barrier that follows decide_pivot: rows
// j..l-1 of the pivot column, as its owner published it (tagged words), into
// xv.  False (and st.stop = 2, the abort flag raised) if a word never became
// fresh.
template <int kThreadsPerCta, typename real>
__device__ __forceinline__ bool fetch_pivot(const CpqrParams<real>& P, int j, int owner, real* xv,
                                            StepState<real>& st) {
  constexpr int W = Words<real>::W;
  const int tid = threadIdx.x, l = P.l;
  const unsigned long long* src = slot_of(P, j & 1, owner);
  const unsigned tag = tag_of(P.gen, j + 1);
  // st.stale was cleared by decide_pivot before the barrier that precedes this
  for (int r = j + tid; r < l; r += kThreadsPerCta) {
    real v;
    if (!get_tagged<real>(src + (int64_t)r * W, tag, &v, P.abort_flag, P.spin)) {
      st.stale = 1;
      v = real(0);
    }
    xv[r] = v;
  }
  cta_sync();
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

// Closing exchange after k_done steps (all threads; S already written): each
// CTA publishes its count of unselected columns, takes the prefix over the
// lower CTAs and writes its unselected columns, ascending, after the pivots
// in J; CTA 0 records k_done and the numerical rank in the status block.
template <typename real>
__device__ __forceinline__ void finish_order(const CpqrParams<real>& P, const int* active, int ncl,
                                             int c0, int k_done, int k_eff, StepState<real>& st) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x, b = blockIdx.x;
  const int fbf = (k_done + 1) & 1;
  const unsigned fep = tag_of(P.gen, k_done + 2);
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
      st.prefix = pre;
      st.stop = ok ? 0 : 2;
      if (!ok) set_flag(&P.status->flags, FLAG_TIMEOUT);
    }
  }
  __syncthreads();
  if (st.stop) return;
  if (tid == 0) {
    int pos = k_done + st.prefix;
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

// Numerical rank: the first step whose pivot norm is zero or at most
// rank_rtol times the first pivot norm (Section 2.3's singular S11).
template <typename real>
__device__ __forceinline__ void note_rank(const CpqrParams<real>& P, int j, real nu, real& nu_first,
                                          int& k_eff) {
  if (j == 0) nu_first = nu;
  if (k_eff < 0 && (nu == real(0) || nu <= P.rank_rtol * nu_first)) {
    k_eff = j;
    if (blockIdx.x == 0 && threadIdx.x == 0) set_flag(&P.status->flags, FLAG_RANK_DEFICIENT);
  }
}

// On return lane t holds the warp-wide sum of a_c for c = (t >> 3) & 3:
// the exchange at offset 16 splits the columns {0,1} / {2,3} between the
// lane halves, the one at offset 8 splits each pair, and three xor rounds
// finish each sum inside its group of 8 lanes.
template <typename real>
__device__ __forceinline__ real reduce4(real a0, real a1, real a2, real a3, int lane) {
  const bool hi = (lane & 16) != 0;
  const real k0 = (hi ? a2 : a0) + __shfl_xor_sync(0xffffffffu, hi ? a0 : a2, 16);
  const real k1 = (hi ? a3 : a1) + __shfl_xor_sync(0xffffffffu, hi ? a1 : a3, 16);
  const bool mid = (lane & 8) != 0;
  real m = (mid ? k1 : k0) + __shfl_xor_sync(0xffffffffu, mid ? k0 : k1, 8);
  m += __shfl_xor_sync(0xffffffffu, m, 4);
  m += __shfl_xor_sync(0xffffffffu, m, 2);
  m += __shfl_xor_sync(0xffffffffu, m, 1);
  return m;
}

// (na, ia) beats (nb, ib) among local columns: ib < 0 is no column; larger
// norm, then smaller index.  A NaN norm never beats a column (the record
// flags it as non-finite instead).
template <typename real>
__device__ __forceinline__ bool local_better(real na, int ia, real nb, int ib) {
  if (ia < 0) return false;
  if (ib < 0) return true;
  if (na > nb) return true;
  return na == nb && ia < ib;
}

template <typename real>
struct WarpBest {
  real bn[kWarps];
  real ss[kWarps];
  int bi[kWarps];
  int nf[kWarps];
};

// Householder reflector of step j from the pivot column x (rows j..l-1) and
// its norm nu: H = I - tau v v^T, v(j) = 1, v(r) = scale x(r) for r > j,
// H x = beta e_j with beta = -sign(x(j)) nu.  nu = 0 gives H = I.
template <typename real>
__device__ __forceinline__ void reflector(real alpha, real nu, real* beta, real* tau, real* scale) {
  *beta = alpha >= real(0) ? -nu : nu;
  *tau = real(0);
  *scale = real(0);
  if (nu > real(0)) {
    *tau = (*beta - alpha) / *beta;
    *scale = real(1) / (alpha - *beta);
  }
}

// Every thread of a CTA, after the barrier that ends fetch_pivot: the
// reflector of step j.  In float64 its two divisions run at a 64th of the
// float32 rate on GB300, so one thread forms it and the CTA shares it
// (one more barrier); in float32 every thread forms its own copy.
template <typename real>
__device__ __forceinline__ void step_reflector(const real* xv, int j, real nu, StepState<real>& st,
                                               real* beta, real* tau, real* scale) {
  if constexpr (sizeof(real) == 8) {
    if (threadIdx.x == 0) reflector(xv[j], nu, &st.beta, &st.tau, &st.scale);
    cta_sync();
    *beta = st.beta;
    *tau = st.tau;
    *scale = st.scale;
  } else {
    reflector(xv[j], nu, beta, tau, scale);
  }
}

// The register-resident kernel (cpqr_reg.cu): whether it takes an l-row
// factorization with nc columns per CTA, and its launch (scratch already
// reset by the caller).
// most columns of a register-resident slab of CTAs with `warps` warps (0: l
// too large), and whether an nc-column slab fits
template <typename real>
int cpqr_reg_cols(int l, int warps);
template <typename real>
bool cpqr_reg_fits(const Ctx& ctx, int l, int nc, int warps);
template <typename real>
curid_status cpqr_reg_launch(const Ctx& ctx, const CpqrParams<real>& P, int G);

}  // namespace cpqr_x

}  // namespace curid
