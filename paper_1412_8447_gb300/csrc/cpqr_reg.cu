// Truncated column-pivoted Householder QR (Section 2.2, Eq. (2.4)-(2.5)) with
// the column slab held in registers: the variant cpqr_run picks when the
// matrix has at most 256 rows (128 in float64) and a CTA's slab at most 64
// columns (the sketch Y = Omega A of Algorithms 1 and 4 and the C^* of
// Algorithm 2 at the ranks of the paper's experiments).
//
// Same grid-wide exchange as the shared-memory kernel (cpqr_exchange.cuh):
// one persistent CTA per SM, one record per CTA and step, tagged candidate
// columns, the pivot column read by every CTA.  What changes is the update:
// warp w keeps slab columns w, w + 16, w + 32, w + 48 for the whole
// factorization, lane t holding rows t, t + 32, ..., t + 32 (RPL - 1) of
// each (rows past l are zero), so a step moves no slab data through shared
// memory.  Each lane builds its rows of the reflector v from the pivot
// column once per step, with v = 0 above row j and v(j) = 1, so neither the
// dot products nor the update need a row mask; the four dot products of a
// warp are summed by one transpose-and-reduce butterfly (10 shuffles instead
// of 4 x 5 plus broadcast); the residual norms are recomputed from rows
// j+1..l-1 like the shared-memory kernel's.  Each warp then posts its best
// column; the CTA's candidate is written to the exchange straight from the
// registers of the warp that holds it.  Measured on the 210 x 6000 and
// 200 x 8000 factorizations of the randomized CUR: 0.929 / 0.935 ms against
// 0.975 / 0.980 ms for the shared-memory kernel (median of 20 launches).
// Variants that were slower: 8 warps of 8 columns (the per-warp dependency
// chains stop overlapping), the owner publishing the reflector (a longer
// publish), reading the best candidate's column while the records come in
// (longer polling rounds).
#include "cpqr_exchange.cuh"

namespace curid {
namespace cpqr_x {

namespace {

constexpr int kMaxCols = 8;                    // columns a warp holds (at most)
constexpr int kMaxRegCols = kWarps * kMaxCols;  // columns of a slab

// Rows a lane can hold for four columns without spilling: 8 per lane in
// float32, 4 in float64 (128 registers per thread at 512 threads).
template <typename real>
constexpr int max_reg_rows() {
  return sizeof(real) == 4 ? 256 : 128;
}

// Each warp, after its residual norms are summed by reduce4 per group of four
// columns (lane t holds the squared norm of column 4 g + ((t >> 3) & 3) in
// qg[g]): post the warp's best unselected column, the sum of its squared
// norms and whether one is not finite.
template <int KC, int NW, typename real>
__device__ __forceinline__ void post_warp_best(const real (&qg)[KC / 4], unsigned act, int lane,
                                               int warp, WarpBest<real>& wb) {
  const int cs = (lane >> 3) & 3;
  real bn = real(-1), ss = real(0);
  int bi = -1, nf = 0;
#pragma unroll
  for (int g = 0; g < KC / 4; ++g) {
    const int c = 4 * g + cs;
    if (!((act >> c) & 1u)) continue;
    const real nv = sqrt(qg[g]);
    ss += nv * nv;
    if (!isfinite(nv)) nf = 1;
    else if (local_better(nv, warp + NW * c, bn, bi)) { bn = nv; bi = warp + NW * c; }
  }
#pragma unroll
  for (int o = 8; o <= 16; o <<= 1) {
    const real on2 = __shfl_xor_sync(0xffffffffu, bn, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (local_better(on2, oi, bn, bi)) { bn = on2; bi = oi; }
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    nf |= __shfl_xor_sync(0xffffffffu, nf, o);
  }
  if (lane == 0) {
    wb.bn[warp] = bn;
    wb.bi[warp] = bi;
    wb.ss[warp] = ss;
    wb.nf[warp] = nf;
  }
}

// Every warp, after the barrier that follows post_warp_best: the CTA's
// candidate for epoch `epoch`.  Warp 0 publishes the record in buffer bf; the
// warp holding the candidate writes its rows r0..l-1 to the CTA's data slot
// as tagged words (readers check every word's tag, so the two writes need no
// order between them).
template <int RPL, int KC, int NW, typename real>
__device__ __forceinline__ void publish_reg(const CpqrParams<real>& P, const WarpBest<real>& wb,
                                            const real (&y)[KC][RPL], int c0, int r0, int bf,
                                            unsigned epoch, int lane, int warp) {
  real bn = lane < NW ? wb.bn[lane] : real(-1);
  int bi = lane < NW ? wb.bi[lane] : -1;
  int nf = lane < NW ? wb.nf[lane] : 0;
#pragma unroll
  for (int o = 1; o < NW; o <<= 1) {
    const real on = __shfl_xor_sync(0xffffffffu, bn, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (local_better(on, oi, bn, bi)) { bn = on; bi = oi; }
    nf |= __shfl_xor_sync(0xffffffffu, nf, o);
  }
  // lanes 0..15 agree; take lane 0's view everywhere
  bn = __shfl_sync(0xffffffffu, bn, 0);
  bi = __shfl_sync(0xffffffffu, bi, 0);
  nf = __shfl_sync(0xffffffffu, nf, 0);
  const unsigned tag = tag_of(P.gen, (int)epoch);
  if (warp == 0) {
    real ss = lane < NW ? wb.ss[lane] : real(0);
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) {
      unsigned hi, lo;
      norm_words<real>(bi >= 0 ? bn : real(0), &hi, &lo);
      const unsigned col = nf ? kNonFinite : (bi >= 0 ? (unsigned)(c0 + bi) : kNoCol);
      st_rec(P.recs + (size_t)bf * gridDim.x + blockIdx.x, pack(tag, col), pack(tag, hi),
             pack(tag, lo), pack(tag, __float_as_uint((float)ss)));
    }
  }
  if (bi >= 0 && !nf && bi % NW == warp) {
    constexpr int W = Words<real>::W;
    unsigned long long* dst = slot_of(P, bf, blockIdx.x);
    const int cb = bi / NW;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      if (c != cb) continue;
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const int r = lane + 32 * u;
        if (r >= r0 && r < P.l) put_tagged<real>(dst + (int64_t)r * W, tag, y[c][u]);
      }
    }
  }
}

template <typename real, int RPL, int KC, int NW>
__global__ void __launch_bounds__(NW * 32, 16 / NW) cpqr_reg_kernel(CpqrParams<real> P) {
  constexpr int NG = KC / 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x;
  const int nc = P.nc, ldl = P.ldl, l = P.l;
  real* ys = reinterpret_cast<real*>(smem_raw);  // nc x ldl staging: input, then S
  real* xv = ys + (int64_t)nc * ldl;             // pivot column of the step
  int* active = reinterpret_cast<int*>(xv + ldl);

  __shared__ StepState<real> st;
  __shared__ WarpBest<real> wb;

  const int c0 = b * nc;
  const int ncl = max(0, min(nc, P.n - c0));

  for (int64_t e = tid; e < (int64_t)l * ncl; e += NW * 32) {
    const int r = (int)(e / ncl), lc = (int)(e % ncl);
    ys[(int64_t)lc * ldl + r] = P.Y[(int64_t)r * P.ldy + c0 + lc];
  }
  for (int lc = tid; lc < nc; lc += NW * 32) active[lc] = lc < ncl ? 1 : 0;
  __syncthreads();

  real y[KC][RPL];
  unsigned act = 0;  // bit c: column warp + 16 c is unselected (warp-uniform)
  {
    real q[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const int lc = warp + NW * c;
      if (lc < ncl) act |= 1u << c;
      q[c] = real(0);
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const int r = lane + 32 * u;
        y[c][u] = (lc < ncl && r < l) ? ys[(int64_t)lc * ldl + r] : real(0);
        q[c] += y[c][u] * y[c][u];
      }
    }
    real qg[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g)
      qg[g] = reduce4(q[4 * g], q[4 * g + 1], q[4 * g + 2], q[4 * g + 3], lane);
    post_warp_best<KC, NW>(qg, act, lane, warp, wb);
  }
  __syncthreads();
  publish_reg<RPL, KC, NW>(P, wb, y, c0, 0, 0, 1u, lane, warp);

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
    if (!fetch_pivot<NW * 32>(P, j, owner, xv, st)) break;
    real beta, tau, scale;
    step_reflector(xv, j, nu, st, &beta, &tau, &scale);
    // v of this lane's rows: 0 above j, 1 at j, scale x(r) below
    real v[RPL];
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      const int r = lane + 32 * u;
      const real x = (r > j && r < l) ? xv[r] : real(0);
      v[u] = r == j ? real(1) : scale * x;
    }
    // dot products (a selected column is zero from row j on, so it needs no
    // mask); with eight columns a warp skips the row blocks of 32 above the
    // pivot row (v is zero there), a warp-uniform branch per block
    real d[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) d[c] = real(0);
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      if (KC > 4 && 32 * u + 31 < j) continue;
#pragma unroll
      for (int c = 0; c < KC; ++c) d[c] += v[u] * y[c][u];
    }
    real dg[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g)
      dg[g] = reduce4(d[4 * g], d[4 * g + 1], d[4 * g + 2], d[4 * g + 3], lane);
    // the warp holding the pivot column retires it: beta at row j, zeros below
    const int pl = pcol - c0;
    const int pc = (pl >= 0 && pl < ncl && pl % NW == warp) ? pl / NW : -1;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      if (c == pc) {
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int r = lane + 32 * u;
          if (r >= j) y[c][u] = r == j ? beta : real(0);
        }
        act &= ~(1u << c);
        if (lane == 0) {
          active[pl] = 0;
          P.J[j] = pcol;
        }
      }
    }
    real q[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      q[c] = real(0);
      const real w = tau * __shfl_sync(0xffffffffu, dg[c / 4], 8 * (c % 4));
      if ((act >> c) & 1u) {
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          if (KC > 4 && 32 * u + 31 < j) continue;
          const int r = lane + 32 * u;
          y[c][u] -= w * v[u];
          if (r > j) q[c] += y[c][u] * y[c][u];
        }
      }
    }
    real qg[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g)
      qg[g] = reduce4(q[4 * g], q[4 * g + 1], q[4 * g + 2], q[4 * g + 3], lane);
    post_warp_best<KC, NW>(qg, act, lane, warp, wb);
    __syncthreads();
    publish_reg<RPL, KC, NW>(P, wb, y, c0, j + 1, (j + 1) & 1, (unsigned)(j + 2), lane, warp);
  }
  const int k_done = j;
  if (st.stop == 2) return;  // timed out: leave without further waits
  // S rows 0..k_done-1 in original column order, staged through shared memory
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    const int lc = warp + NW * c;
    if (lc < ncl) {
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const int r = lane + 32 * u;
        if (r < k_done) ys[(int64_t)lc * ldl + r] = y[c][u];
      }
    }
  }
  __syncthreads();
  for (int64_t e = tid; e < (int64_t)k_done * ncl; e += NW * 32) {
    const int i = (int)(e / ncl), lc = (int)(e % ncl);
    P.S[(int64_t)i * P.lds + c0 + lc] = ys[(int64_t)lc * ldl + i];
  }
  finish_order(P, active, ncl, c0, k_done, k_eff, st);
}

template <typename real>
size_t reg_smem_bytes(int nc, int ldl) {
  return (size_t)nc * ldl * sizeof(real) + (size_t)ldl * sizeof(real) + (size_t)nc * sizeof(int) +
         16;
}

}  // namespace

// Eight columns per warp fit the registers without spilling up to 224 rows
// in float32 and 64 in float64; four up to 256 / 128 rows.
template <typename real>
int cpqr_reg_cols(int l, int warps) {
  if (l < 1 || l > max_reg_rows<real>()) return 0;
  const int wide_rows = sizeof(real) == 4 ? 224 : 64;
  return warps * (l <= wide_rows ? 8 : 4);
}

template <typename real>
bool cpqr_reg_fits(const Ctx& ctx, int l, int nc, int warps) {
  // the kernel's static shared variables share the per-block limit
  return nc >= 1 && nc <= cpqr_reg_cols<real>(l, warps) &&
         reg_smem_bytes<real>(nc, l | 1) + 1024 <= ctx.smem_optin;
}

namespace {

template <typename real, int NW>
void (*reg_kernel_for(int l, int nc))(CpqrParams<real>) {
  const bool wide = nc > NW * 4;
  if (l <= 64) return wide ? cpqr_reg_kernel<real, 2, 8, NW> : cpqr_reg_kernel<real, 2, 4, NW>;
  if (l <= 128) {
    if constexpr (sizeof(real) == 4)
      return wide ? cpqr_reg_kernel<real, 4, 8, NW> : cpqr_reg_kernel<real, 4, 4, NW>;
    else
      return cpqr_reg_kernel<real, 4, 4, NW>;
  }
  if constexpr (sizeof(real) == 4) {
    if (l <= 224) return wide ? cpqr_reg_kernel<real, 7, 8, NW> : cpqr_reg_kernel<real, 7, 4, NW>;
    return cpqr_reg_kernel<real, 8, 4, NW>;
  }
  return nullptr;
}

}  // namespace

template <typename real>
curid_status cpqr_reg_launch(const Ctx& ctx, const CpqrParams<real>& P, int G) {
  const int warps = kWarps;
  if (P.warps != warps || !cpqr_reg_fits<real>(ctx, P.l, P.nc, warps)) return CURID_UNSUPPORTED;
  const size_t smem = reg_smem_bytes<real>(P.nc, P.ldl);
  void (*fn)(CpqrParams<real>) = reg_kernel_for<real, kWarps>(P.l, P.nc);
  if (!fn) return CURID_UNSUPPORTED;
  CURID_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CpqrParams<real> Pc = P;
  void* args[] = {&Pc};
  CURID_CUDA(cudaLaunchCooperativeKernel((void*)fn, dim3(G), dim3(warps * 32), args, smem,
                                         ctx.stream));
  if (ctx.launches) ++*ctx.launches;
  return CURID_OK;
}

template int cpqr_reg_cols<float>(int, int);
template int cpqr_reg_cols<double>(int, int);
template bool cpqr_reg_fits<float>(const Ctx&, int, int, int);
template bool cpqr_reg_fits<double>(const Ctx&, int, int, int);
template curid_status cpqr_reg_launch<float>(const Ctx&, const CpqrParams<float>&, int);
template curid_status cpqr_reg_launch<double>(const Ctx&, const CpqrParams<double>&, int);

}  // namespace cpqr_x
}  // namespace curid
