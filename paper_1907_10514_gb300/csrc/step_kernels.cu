// step_kernels.cu -- the fused timestep kernels of libiontrap.so (sm_103a).
//
// One launch = one velocity-Verlet step for one simulation (Sec. 6 "Integration"):
//   grid.x : i-blocks of T*I ions (I ions per thread, in registers)
//   grid.y : splits of the j-range, jsplit ions each, staged into shared memory by one
//            bulk TMA copy per stream (hi and lo), completing on an mbarrier
// Every CTA sums the Coulomb term (Eq. 4, direct sum, Sec. 6 "Interactions") of its
// i-block over its j-range and writes the partial to scratch.  The last CTA to finish
// an i-block (arrival counter) merges the partials in split order and runs the fused
// epilogue: trap field (Eq. 1/3) + Langevin bath (Sec. 3) + Verlet kick/drift, and
// writes the next pair stream.  The last i-block to finish advances the device step
// counter, so a chain of launches (a CUDA graph) needs no host round trip.
//
// Summation order is a function of (n, T, I, jsplit) only: j ascending inside each
// 128-wide segment (plain FP32), segments Kahan-added per CTA, CTA partials merged in
// split order.  The same configuration always gives the same bits.
#include <cooperative_groups.h>

#include <cstdio>

#include "iontrap_internal.cuh"

namespace cg = cooperative_groups;

namespace it {

// Programmatic dependent launch: let the next step's CTAs be scheduled as this grid's
// CTAs retire, and wait for the previous step's grid (its memory included) before
// touching any state.  Both are no-ops for a launch without the PDL attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Stage a whole j-range (bytes per stream) with bulk TMA; every thread waits with a
// time limit.  Returns false (error flag set, copies drained) if the wait expired.
__device__ __forceinline__ bool stage_jrange(uint64_t* bar, void* d0, const void* s0, void* d1, const void* s1,
                                             uint32_t bytes, int* err) {
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, s1 ? 2u * bytes : bytes);
    tma_bulk_g2s(d0, s0, bytes, bar);
    if (s1) tma_bulk_g2s(d1, s1, bytes, bar);
  }
  const bool ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicOr(err, ERR_TIMEOUT);
      mbar_wait_bounded(bar, 0, kWaitLimitNs);
    }
    __syncthreads();
    return false;
  }
  return true;
}

// Arrival at the i-block counter; true in the last CTA of the i-block.
__device__ __forceinline__ bool arrive_last(unsigned* cnt, unsigned expected, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(cnt, 1u);
    *s_flag = (prev == expected - 1u);
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// Reset the i-block counter and, in the last i-block, advance the step counter.
__device__ __forceinline__ void finish_iblock(const StepArgs& A, long long ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    A.cnt[blockIdx.x] = 0u;
    __threadfence();
    const unsigned prev = atomicAdd(A.done, 1u);
    if (prev == gridDim.x - 1u) {
      *A.done = 0u;
      if (A.mode == MODE_STEP) *A.step = ns + 1;
      __threadfence();
    }
  }
}

__device__ __forceinline__ void merge_f64(const double4_32a* __restrict__ part, long long n, long long i,
                                          int nsplit, double S[3]) {
  double s[3] = {0.0, 0.0, 0.0};
  for (int p = 0; p < nsplit; ++p) {
    const double2* r = reinterpret_cast<const double2*>(part + p * n + i);
    const double2 xy = __ldcg(r), zw = __ldcg(r + 1);
    s[0] += xy.x;
    s[1] += xy.y;
    s[2] += zw.x;
  }
  S[0] = s[0], S[1] = s[1], S[2] = s[2];
}

// ------------------------------------------------------------------ FP32 form
constexpr int kChunk = kSeg;  // j-chunk staged per TMA transaction = one Kahan segment

// The pair sum of one CTA: its i-block (T*I ions, I per thread in registers) against
// its j-range [j0, j1), staged in 128-ion chunks by double-buffered bulk TMA.  Leaves
// the per-thread Kahan pairs (ks, kc) -- negated sums -- and returns false if a staged
// chunk never arrived (error flag set, copies drained).
template <int T, int I, bool PACK>
__device__ __forceinline__ bool pair_sums(const StepArgs& A, float4 (&sh)[2][kChunk], float4 (&sl)[2][kChunk],
                                          uint64_t (&bar)[2], const float4* __restrict__ ghi,
                                          const float4* __restrict__ glo, long long i0, long long j0, long long j1,
                                          float (&ks)[I][3], float (&kc)[I][3]) {
  const int tid = threadIdx.x;
  const long long n = A.n;
  const int nch = (int)((j1 - j0 + kChunk - 1) / kChunk);
  const bool coulomb = !(A.trap.flags & IONTRAP_COULOMB_OFF);
  if (coulomb) {
    auto issue = [&](int c) {
      const long long jc = j0 + (long long)c * kChunk;
      const uint32_t bytes = (uint32_t)min((long long)kChunk, j1 - jc) * 16u;
      const int b = c & 1;
      mbar_arrive_expect_tx(&bar[b], 2u * bytes);
      tma_bulk_g2s(sh[b], ghi + jc, bytes, &bar[b]);
      tma_bulk_g2s(sl[b], glo + jc, bytes, &bar[b]);
    };
    if (tid == 0) {
      mbar_init(&bar[0], 1);
      mbar_init(&bar[1], 1);
    }
    __syncthreads();
    if (tid == 0) {
      issue(0);
      if (nch > 1) issue(1);
    }
    long long ii[I];
    float nxh[I][3], nxl[I][3];
#pragma unroll
    for (int k = 0; k < I; ++k) {
      ii[k] = i0 + k * T + tid;
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
      if (ii[k] < n) {
        h = ghi[ii[k]];
        l = glo[ii[k]];
      }
      nxh[k][0] = -h.x, nxh[k][1] = -h.y, nxh[k][2] = -h.z;
      nxl[k][0] = -l.x, nxl[k][1] = -l.y, nxl[k][2] = -l.z;
    }
    const long long iend = i0 + T * I;
    for (int c = 0; c < nch; ++c) {
      const int b = c & 1;
      const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((c >> 1) & 1), kWaitLimitNs);
      const long long jc = j0 + (long long)c * kChunk;
      const int jn = (int)min((long long)kChunk, j1 - jc);
      const bool diag = (jc < iend) && (i0 < jc + jn);
      float acc[I][3];
      if constexpr (PACK) {
        float2 nxh2[I / 2][3], nxl2[I / 2][3], acc2[I / 2][3];
#pragma unroll
        for (int k = 0; k < I / 2; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            nxh2[k][d] = make_float2(nxh[2 * k][d], nxh[2 * k + 1][d]);
            nxl2[k][d] = make_float2(nxl[2 * k][d], nxl[2 * k + 1][d]);
            acc2[k][d] = make_float2(0.0f, 0.0f);
          }
        if (A.unitw) {
          if (diag)
            segment_f32x2<I, true, true>(sh[b], sl[b], jn, jc, nxh2, nxl2, ii, acc2);
          else
            segment_f32x2<I, false, true>(sh[b], sl[b], jn, jc, nxh2, nxl2, ii, acc2);
        } else {
          if (diag)
            segment_f32x2<I, true>(sh[b], sl[b], jn, jc, nxh2, nxl2, ii, acc2);
          else
            segment_f32x2<I, false>(sh[b], sl[b], jn, jc, nxh2, nxl2, ii, acc2);
        }
#pragma unroll
        for (int k = 0; k < I / 2; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            acc[2 * k][d] = acc2[k][d].x;
            acc[2 * k + 1][d] = acc2[k][d].y;
          }
      } else {
#pragma unroll
        for (int k = 0; k < I; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) acc[k][d] = 0.0f;
        if (A.unitw) {
          if (diag)
            segment_f32<I, true, true>(sh[b], sl[b], jn, jc, nxh, nxl, ii, acc);
          else
            segment_f32<I, false, true>(sh[b], sl[b], jn, jc, nxh, nxl, ii, acc);
        } else {
          if (diag)
            segment_f32<I, true>(sh[b], sl[b], jn, jc, nxh, nxl, ii, acc);
          else
            segment_f32<I, false>(sh[b], sl[b], jn, jc, nxh, nxl, ii, acc);
        }
      }
      // Kahan: value = ks - kc
#pragma unroll
      for (int k = 0; k < I; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float y = acc[k][d] - kc[k][d];
          const float t = ks[k][d] + y;
          kc[k][d] = (t - ks[k][d]) - y;
          ks[k][d] = t;
        }
      if (__syncthreads_or(!ok)) {  // a staged chunk never arrived: drain and give up
        if (tid == 0) {
          atomicOr(A.err, ERR_TIMEOUT);
          for (int q = c; q < min(c + 2, nch); ++q)
            mbar_wait_bounded(&bar[q & 1], (uint32_t)((q >> 1) & 1), kWaitLimitNs);
        }
        __syncthreads();
        return false;
      }
      if (tid == 0 && c + 2 < nch) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(c + 2);
      }
    }
  }

  return true;
}

template <int T, int I, bool PACK, bool FUSED>
__global__ void __launch_bounds__(T) k_step_f32(const __grid_constant__ StepArgs A) {
  __shared__ __align__(128) float4 sh[2][kChunk];
  __shared__ __align__(128) float4 sl[2][kChunk];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_flag;
  __shared__ double s_cos;
  __shared__ double s_springs[IONTRAP_MAX_SPECIES][3];

  pdl_wait();
  const int tid = threadIdx.x;
  const long long n = A.n;
  const long long i0 = (long long)blockIdx.x * (T * I);
  const long long j0 = (long long)blockIdx.y * A.jsplit;
  const long long j1 = min(j0 + (long long)A.jsplit, n);
  const long long ns = *A.step;
  const int rb = (A.mode == MODE_STEP) ? (int)((ns + 1) & 1) : (int)(ns & 1);
  const float4* __restrict__ ghi = A.hi[rb];
  const float4* __restrict__ glo = A.lo[rb];
  const long long tslot = 4ll * (blockIdx.y * (long long)gridDim.x + blockIdx.x);
  trace_mark(A.trace, tslot + 0);

  float ks[I][3], kc[I][3];
#pragma unroll
  for (int k = 0; k < I; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) ks[k][c] = kc[k][c] = 0.0f;

  if (!pair_sums<T, I, PACK>(A, sh, sl, bar, ghi, glo, i0, j0, j1, ks, kc)) return;

  trace_mark(A.trace, tslot + 1);
  pdl_trigger();  // dependents launch as the last CTAs finish their pair loops
  float4* part = reinterpret_cast<float4*>(A.part);
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const long long i = i0 + k * T + tid;
    if (i < n) {
      const long long r = 2 * (blockIdx.y * n + i);
      __stcg(part + r, make_float4(ks[k][0], ks[k][1], ks[k][2], 0.0f));
      __stcg(part + r + 1, make_float4(kc[k][0], kc[k][1], kc[k][2], 0.0f));
    }
  }
  if constexpr (!FUSED) return;  // the epilogue kernel merges the partials
  if (!arrive_last(&A.cnt[blockIdx.x], gridDim.y, &s_flag)) return;
  trace_mark(A.trace, tslot + 2);

  if (tid == 0) s_cos = force_time_cos(A, ns);
  __syncthreads();
  if (tid < IONTRAP_MAX_SPECIES) trap_springs(A.trap, A.spc[tid], s_cos, s_springs[tid]);
  __syncthreads();
  const int wb = rb ^ 1;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const long long i = i0 + k * T + tid;
    if (i >= n) continue;
    double S[3];
    merge_f32(part, n, i, (int)gridDim.y, S);  // fused path: the last CTA of the i-block
    epilogue_ion<false>(A, i, S, s_springs, ns, wb);
  }
  finish_iblock(A, ns);
  trace_mark(A.trace, tslot + 3);
}

// Cluster form: the S CTAs that sum one i-block over the S j-splits (grid.y = S <= 8)
// are one thread-block cluster.  Each CTA leaves its (sum, compensation) pairs in its
// shared memory; after a cluster barrier, CTA r merges ions [r*B/S, (r+1)*B/S) of the
// i-block (B = T*I) by reading the S partials through distributed shared memory in
// split order, and integrates them.  No global partials, no arrival counters, and the
// FP64 epilogue is spread over S SMs.  Same merge order as the other forms: identical
// bits for an equal (T*I, jsplit).
template <int T, int I, bool PACK>
__global__ void __launch_bounds__(T) k_step_f32_cl(const __grid_constant__ StepArgs A) {
  __shared__ __align__(128) float4 sh[2][kChunk];
  __shared__ __align__(128) float4 sl[2][kChunk];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ __align__(16) float4 s_part[T * I][2];
  __shared__ double s_cos;
  __shared__ double s_springs[IONTRAP_MAX_SPECIES][3];
  cg::cluster_group cluster = cg::this_cluster();

  pdl_wait();
  const int tid = threadIdx.x;
  const long long n = A.n;
  const long long i0 = (long long)blockIdx.x * (T * I);
  const long long j0 = (long long)blockIdx.y * A.jsplit;
  const long long j1 = min(j0 + (long long)A.jsplit, n);
  const long long ns = *A.step;
  const int rb = (A.mode == MODE_STEP) ? (int)((ns + 1) & 1) : (int)(ns & 1);
  const long long tslot = 4ll * (blockIdx.y * (long long)gridDim.x + blockIdx.x);
  trace_mark(A.trace, tslot + 0);
  if (tid == 0) s_cos = force_time_cos(A, ns);

  float ks[I][3], kc[I][3];
#pragma unroll
  for (int k = 0; k < I; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) ks[k][c] = kc[k][c] = 0.0f;
  // on an expired wait the error flag is set and the CTA still meets every cluster
  // barrier below (the result of this step is then discarded by the caller)
  pair_sums<T, I, PACK>(A, sh, sl, bar, A.hi[rb], A.lo[rb], i0, j0, j1, ks, kc);
  trace_mark(A.trace, tslot + 1);
  pdl_trigger();
#pragma unroll
  for (int k = 0; k < I; ++k) {
    s_part[k * T + tid][0] = make_float4(ks[k][0], ks[k][1], ks[k][2], 0.0f);
    s_part[k * T + tid][1] = make_float4(kc[k][0], kc[k][1], kc[k][2], 0.0f);
  }
  __syncthreads();  // s_cos
  if (tid < IONTRAP_MAX_SPECIES) trap_springs(A.trap, A.spc[tid], s_cos, s_springs[tid]);
  cluster.sync();  // every CTA's partials written; springs ready
  trace_mark(A.trace, tslot + 2);

  const int S = (int)gridDim.y;
  const int r = (int)cluster.block_rank();
  constexpr int B = T * I;
  const int per = (B + S - 1) / S;
  for (int q = r * per + tid; q < min(B, (r + 1) * per); q += T) {
    const long long i = i0 + q;
    if (i >= n) continue;
    float4 pa[8], pc[8];
#pragma unroll
    for (int p = 0; p < 8; ++p)
      if (p < S) {
        const float4* rec = cluster.map_shared_rank(&s_part[q][0], (unsigned)p);
        pa[p] = rec[0];
        pc[p] = rec[1];
      }
    float su[3] = {0.f, 0.f, 0.f}, cu[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int p = 0; p < 8; ++p)
      if (p < S) {
        kahan_merge(su[0], cu[0], pa[p].x, pc[p].x);
        kahan_merge(su[1], cu[1], pa[p].y, pc[p].y);
        kahan_merge(su[2], cu[2], pa[p].z, pc[p].z);
      }
    double Sd[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Sd[c] = (double)cu[c] - (double)su[c];
    epilogue_ion<false>(A, i, Sd, s_springs, ns, rb ^ 1);
  }
  trace_mark(A.trace, tslot + 3);
  cluster.sync();  // no CTA leaves while another may still read its partials
  if (r == 0 && tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(A.done, 1u);
    if (prev == gridDim.x - 1u) {
      *A.done = 0u;
      if (A.mode == MODE_STEP) *A.step = ns + 1;
      __threadfence();
    }
  }
}

// Cluster + warp-split form (fused = 3): the i-block is 32*I ions (I per lane, the same
// ions in every warp); the W warps of a CTA sum interleaved 128-ion chunks of the CTA's
// j-range (warp w takes chunks w, w+W, ...; one bulk TMA per round stages W consecutive
// chunks, double-buffered), their partials are folded in warp order, and the S CTAs of
// an i-block (a cluster, S <= 8) are folded in split order through distributed shared
// memory.  The part of each ion's epilogue that does not depend on the Coulomb sum
// (kick, drift, trap, drag, noise) is evaluated before the pair loop, so after the
// final fold only the last few FP64 operations remain.
template <int I, int W, bool PACK>
__global__ void __launch_bounds__(32 * W) k_step_f32_cw(const __grid_constant__ StepArgs A) {
  constexpr int T = 32 * W;
  constexpr int B = 32 * I;
  static_assert(W * kChunk * 64 + W * B * 32 + B * 32 <= 47 * 1024, "static shared memory above the 48 KB limit");
  __shared__ __align__(128) float4 sh[2][W * kChunk];
  __shared__ __align__(128) float4 sl[2][W * kChunk];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ __align__(16) float4 s_wp[W][B][2];
  __shared__ __align__(16) float4 s_part[B][2];
  __shared__ double s_cos;
  __shared__ double s_springs[IONTRAP_MAX_SPECIES][3];
  cg::cluster_group cluster = cg::this_cluster();

  pdl_wait();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long n = A.n;
  const long long i0 = (long long)blockIdx.x * B;
  const long long j0 = (long long)blockIdx.y * A.jsplit;
  const long long j1 = min(j0 + (long long)A.jsplit, n);
  const long long ns = *A.step;
  const int rb = (A.mode == MODE_STEP) ? (int)((ns + 1) & 1) : (int)(ns & 1);
  const float4* __restrict__ ghi = A.hi[rb];
  const float4* __restrict__ glo = A.lo[rb];
  const long long tslot = 4ll * (blockIdx.y * (long long)gridDim.x + blockIdx.x);
  trace_mark(A.trace, tslot + 0);
  const bool coulomb = !(A.trap.flags & IONTRAP_COULOMB_OFF);
  const int nch = coulomb ? (int)((j1 - j0 + kChunk - 1) / kChunk) : 0;  // nothing staged without the pair term
  const int nr = (nch + W - 1) / W;
  auto issue = [&](int k) {  // round k: chunks kW .. kW+W-1, consecutive in j
    const long long jc = j0 + (long long)k * W * kChunk;
    const uint32_t bytes = (uint32_t)min((long long)W * kChunk, j1 - jc) * 16u;
    const int b = k & 1;
    mbar_arrive_expect_tx(&bar[b], 2u * bytes);
    tma_bulk_g2s(sh[b], ghi + jc, bytes, &bar[b]);
    tma_bulk_g2s(sl[b], glo + jc, bytes, &bar[b]);
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_cos = force_time_cos(A, ns);
  }
  __syncthreads();
  if (tid == 0) {
    if (nr > 0) issue(0);
    if (nr > 1) issue(1);
  }
  if (tid < IONTRAP_MAX_SPECIES) trap_springs(A.trap, A.spc[tid], s_cos, s_springs[tid]);
  __syncthreads();

  // this thread's epilogue ion (CTA r of the cluster integrates a slice of the i-block)
  const int S = (int)gridDim.y;
  const int r = (int)cluster.block_rank();
  const int per = (B + S - 1) / S;
  const int q = r * per + tid;
  const long long ie = i0 + q;
  const bool own = tid < per && q < B && ie < n;
  const bool step = (A.mode == MODE_STEP), forces = (A.mode == MODE_FORCES);
  double xf[3], vd[3], v0[3], ext[3];
  int spe = 0;
  if (own && !forces) {
    spe = A.sp[ie];
    const TrapDev& tp = A.trap;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x = A.x[c * n + ie], v = A.v[c * n + ie], a = A.a[c * n + ie];
      const double vh = half_kick(v, a, tp.hdt);
      v0[c] = v;
      vd[c] = step ? vh : v;
      xf[c] = step ? drift(x, vh, tp.dt) : x;
    }
    accel_ext<false>(tp, A.spc[spe], s_springs[spe], xf, vd, step ? ns + 1 : ns, ie, ext);
  }

  // pair sums of this warp's chunks
  long long ii[I];
  float nxh[I][3], nxl[I][3], ks[I][3], kc[I][3];
#pragma unroll
  for (int k = 0; k < I; ++k) {
    ii[k] = i0 + k * 32 + lane;
    float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
    if (ii[k] < n) {
      h = ghi[ii[k]];
      l = glo[ii[k]];
    }
    nxh[k][0] = -h.x, nxh[k][1] = -h.y, nxh[k][2] = -h.z;
    nxl[k][0] = -l.x, nxl[k][1] = -l.y, nxl[k][2] = -l.z;
#pragma unroll
    for (int c = 0; c < 3; ++c) ks[k][c] = kc[k][c] = 0.0f;
  }
  const long long iend = i0 + B;
  for (int k = 0; k < nr; ++k) {
    const int b = k & 1;
    const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1), kWaitLimitNs);
    const int c = k * W + warp;
    if (c < nch) {
      const long long jc = j0 + (long long)c * kChunk;
      const int jn = (int)min((long long)kChunk, j1 - jc);
      const bool diag = (jc < iend) && (i0 < jc + jn);
      const float4* csh = sh[b] + warp * kChunk;
      const float4* csl = sl[b] + warp * kChunk;
      float acc[I][3];
      if constexpr (PACK) {
        float2 nxh2[I / 2][3], nxl2[I / 2][3], acc2[I / 2][3];
#pragma unroll
        for (int k2 = 0; k2 < I / 2; ++k2)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            nxh2[k2][d] = make_float2(nxh[2 * k2][d], nxh[2 * k2 + 1][d]);
            nxl2[k2][d] = make_float2(nxl[2 * k2][d], nxl[2 * k2 + 1][d]);
            acc2[k2][d] = make_float2(0.0f, 0.0f);
          }
        if (A.unitw) {
          if (diag)
            segment_f32x2<I, true, true>(csh, csl, jn, jc, nxh2, nxl2, ii, acc2);
          else
            segment_f32x2<I, false, true>(csh, csl, jn, jc, nxh2, nxl2, ii, acc2);
        } else {
          if (diag)
            segment_f32x2<I, true>(csh, csl, jn, jc, nxh2, nxl2, ii, acc2);
          else
            segment_f32x2<I, false>(csh, csl, jn, jc, nxh2, nxl2, ii, acc2);
        }
#pragma unroll
        for (int k2 = 0; k2 < I / 2; ++k2)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            acc[2 * k2][d] = acc2[k2][d].x;
            acc[2 * k2 + 1][d] = acc2[k2][d].y;
          }
      } else {
#pragma unroll
        for (int k2 = 0; k2 < I; ++k2)
#pragma unroll
          for (int d = 0; d < 3; ++d) acc[k2][d] = 0.0f;
        if (A.unitw) {
          if (diag)
            segment_f32<I, true, true>(csh, csl, jn, jc, nxh, nxl, ii, acc);
          else
            segment_f32<I, false, true>(csh, csl, jn, jc, nxh, nxl, ii, acc);
        } else {
          if (diag)
            segment_f32<I, true>(csh, csl, jn, jc, nxh, nxl, ii, acc);
          else
            segment_f32<I, false>(csh, csl, jn, jc, nxh, nxl, ii, acc);
        }
      }
#pragma unroll
      for (int k2 = 0; k2 < I; ++k2)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float y = acc[k2][d] - kc[k2][d];
          const float t = ks[k2][d] + y;
          kc[k2][d] = (t - ks[k2][d]) - y;
          ks[k2][d] = t;
        }
    }
    if (__syncthreads_or(!ok)) {  // a staged round never arrived: drain, flag, and still meet the cluster
      if (tid == 0) {
        atomicOr(A.err, ERR_TIMEOUT);
        for (int kk = k; kk < min(k + 2, nr); ++kk)
          mbar_wait_bounded(&bar[kk & 1], (uint32_t)((kk >> 1) & 1), kWaitLimitNs);
      }
      __syncthreads();
      break;
    }
    if (tid == 0 && k + 2 < nr) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(k + 2);
    }
  }
  trace_mark(A.trace, tslot + 1);
  pdl_trigger();
  // fold the warps' partials in warp order
#pragma unroll
  for (int k = 0; k < I; ++k) {
    s_wp[warp][k * 32 + lane][0] = make_float4(ks[k][0], ks[k][1], ks[k][2], 0.0f);
    s_wp[warp][k * 32 + lane][1] = make_float4(kc[k][0], kc[k][1], kc[k][2], 0.0f);
  }
  __syncthreads();
  for (int qq = tid; qq < B; qq += T) {
    float su[3] = {0.f, 0.f, 0.f}, cu[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const float4 pa = s_wp[w][qq][0], pc = s_wp[w][qq][1];
      kahan_merge(su[0], cu[0], pa.x, pc.x);
      kahan_merge(su[1], cu[1], pa.y, pc.y);
      kahan_merge(su[2], cu[2], pa.z, pc.z);
    }
    s_part[qq][0] = make_float4(su[0], su[1], su[2], 0.0f);
    s_part[qq][1] = make_float4(cu[0], cu[1], cu[2], 0.0f);
  }
  cluster.sync();  // every CTA's partials are folded and visible
  trace_mark(A.trace, tslot + 2);
  if (own) {
    float su[3] = {0.f, 0.f, 0.f}, cu[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int p0 = 0; p0 < 16; p0 += 8) {
      if (p0 >= S) break;
      float4 pa[8], pc[8];
#pragma unroll
      for (int p = 0; p < 8; ++p)
        if (p0 + p < S) {
          const float4* rec = cluster.map_shared_rank(&s_part[q][0], (unsigned)(p0 + p));
          pa[p] = rec[0];
          pc[p] = rec[1];
        }
#pragma unroll
      for (int p = 0; p < 8; ++p)
        if (p0 + p < S) {
          kahan_merge(su[0], cu[0], pa[p].x, pc[p].x);
          kahan_merge(su[1], cu[1], pa[p].y, pc[p].y);
          kahan_merge(su[2], cu[2], pa[p].z, pc[p].z);
        }
    }
    double Sd[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Sd[c] = (double)cu[c] - (double)su[c];
    if (forces) {
      const SpeciesDev& sd = A.spc[A.sp[ie]];
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out[c * n + ie] = sd.coul * Sd[c];
    } else {
      const SpeciesDev& sd = A.spc[spe];
      const TrapDev& tp = A.trap;
      double acc[3], vn[3], xn[3];
      accel_total(sd, Sd, ext, acc);
      bool finite = true;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vn[c] = step ? half_kick(vd[c], acc[c], tp.hdt) : v0[c];
        xn[c] = drift(xf[c], half_kick(vn[c], acc[c], tp.hdt), tp.dt);
        finite = finite && isfinite(acc[c]) && isfinite(vn[c]) && isfinite(xn[c]);
        if (step) {
          A.x[c * n + ie] = xf[c];
          A.v[c * n + ie] = vn[c];
        }
        A.a[c * n + ie] = acc[c];
      }
      write_pair<false>(A, rb ^ 1, ie, xn, sd.w);
      if (!finite) atomicOr(A.err, ERR_NONFINITE);
    }
  }
  trace_mark(A.trace, tslot + 3);
  cluster.sync();  // no CTA leaves while another may still read its partials
  if (r == 0 && tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(A.done, 1u);
    if (prev == gridDim.x - 1u) {
      *A.done = 0u;
      if (A.mode == MODE_STEP) *A.step = ns + 1;
      __threadfence();
    }
  }
}

// Separate epilogue over all SMs.  A CTA of 256 threads serves 32 ions: 8 lanes per ion
// fetch the ion's split records together (one memory round trip instead of one per
// split), fold them in split order through warp shuffles, and leave the merged sum in
// shared memory; then one warp integrates the 32 ions, one per lane.  The last CTA
// advances the step counter.
constexpr int kEpiIons = 32;
constexpr int kEpiThreads = 256;
constexpr int kEpiMaxRec = 8;  // records per lane: splits up to 8 * 8 = 64

__global__ void __launch_bounds__(kEpiThreads) k_epilogue_f32(const __grid_constant__ StepArgs A) {
  __shared__ double s_cos;
  __shared__ double s_springs[IONTRAP_MAX_SPECIES][3];
  __shared__ int s_last;
  pdl_wait();
  const long long n = A.n;
  const long long ns = *A.step;
  const int rb = (A.mode == MODE_STEP) ? (int)((ns + 1) & 1) : (int)(ns & 1);
  unsigned long long* et = A.trace ? A.trace + A.trace_epi : nullptr;
  trace_mark(et, 2ll * blockIdx.x);
  if (threadIdx.x == 0) s_cos = force_time_cos(A, ns);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane & 7;                       // lane within the ion's group of 8
  const int slot = warp * 4 + (lane >> 3);        // ion slot in this CTA
  const long long i = blockIdx.x * (long long)kEpiIons + slot;
  const int nsplit = A.nsplit;
  const float4* __restrict__ part = reinterpret_cast<const float4*>(A.part);
  float4 ra[kEpiMaxRec], rc[kEpiMaxRec];
#pragma unroll
  for (int q = 0; q < kEpiMaxRec; ++q) {
    const int p = q * 8 + sub;
    ra[q] = rc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n && p < nsplit) {
      ra[q] = __ldcg(part + 2 * (p * n + i));
      rc[q] = __ldcg(part + 2 * (p * n + i) + 1);
    }
  }
  float s[3] = {0.f, 0.f, 0.f}, cc[3] = {0.f, 0.f, 0.f};
  const int base = lane & ~7;
#pragma unroll
  for (int q = 0; q < kEpiMaxRec; ++q) {
    if (q * 8 >= nsplit) break;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int p = q * 8 + l;  // uniform across the warp
      const float ax = __shfl_sync(0xffffffffu, ra[q].x, base + l), ay = __shfl_sync(0xffffffffu, ra[q].y, base + l);
      const float az = __shfl_sync(0xffffffffu, ra[q].z, base + l), cx = __shfl_sync(0xffffffffu, rc[q].x, base + l);
      const float cy = __shfl_sync(0xffffffffu, rc[q].y, base + l), cz = __shfl_sync(0xffffffffu, rc[q].z, base + l);
      if (p < nsplit) {
        kahan_merge(s[0], cc[0], ax, cx);
        kahan_merge(s[1], cc[1], ay, cy);
        kahan_merge(s[2], cc[2], az, cz);
      }
    }
  }
  pdl_trigger();
  __syncthreads();  // s_cos
  if (threadIdx.x < IONTRAP_MAX_SPECIES) trap_springs(A.trap, A.spc[threadIdx.x], s_cos, s_springs[threadIdx.x]);
  __syncthreads();
  // one lane per ion integrates; the 32 ions are spread over the 8 warps (4 per warp)
  if (sub == 0 && i < n) {
    double S[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) S[c] = (double)cc[c] - (double)s[c];
    epilogue_ion<false>(A, i, S, s_springs, ns, rb ^ 1);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(A.done, 1u);
    s_last = (prev == gridDim.x - 1u);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    *A.done = 0u;
    if (A.mode == MODE_STEP) *A.step = ns + 1;
    __threadfence();
  }
  trace_mark(et, 2ll * blockIdx.x + 1);
}

// ------------------------------------------------------------------ FP64 plain form
template <int I, bool DIAG>
__device__ __forceinline__ void segment_f64(const double4_32a* __restrict__ sp, int g0, int g1, long long jbase,
                                            const double (&xi)[I][3], const long long (&ii)[I],
                                            double (&acc)[I][3]) {
#pragma unroll 2
  for (int j = g0; j < g1; ++j) {
    const double4_32a p = sp[j];
#pragma unroll
    for (int k = 0; k < I; ++k) {
      const double dx = xi[k][0] - p.x;
      const double dy = xi[k][1] - p.y;
      const double dz = xi[k][2] - p.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      double ri = rsqrt(r2);
      if (DIAG) ri = (jbase + j == ii[k]) ? 0.0 : ri;
      const double s = p.w * ri * ri * ri;
      acc[k][0] += s * dx;
      acc[k][1] += s * dy;
      acc[k][2] += s * dz;
    }
  }
}

template <int T, int I>
__global__ void __launch_bounds__(T) k_step_f64(const __grid_constant__ StepArgs A) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_flag;
  __shared__ double s_cos;
  double4_32a* sp = reinterpret_cast<double4_32a*>(smraw);
  __shared__ double s_springs[IONTRAP_MAX_SPECIES][3];

  pdl_wait();
  const int tid = threadIdx.x;
  const long long n = A.n;
  const long long i0 = (long long)blockIdx.x * (T * I);
  const long long j0 = (long long)blockIdx.y * A.jsplit;
  const int jn = (int)min((long long)A.jsplit, n - j0);  // FP64 form: whole j-range staged
  const long long ns = *A.step;
  const int rb = (A.mode == MODE_STEP) ? (int)((ns + 1) & 1) : (int)(ns & 1);
  const bool coulomb = !(A.trap.flags & IONTRAP_COULOMB_OFF);

  double acc[I][3];
#pragma unroll
  for (int k = 0; k < I; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[k][c] = 0.0;

  if (coulomb) {
    if (!stage_jrange(&bar, sp, A.p64[rb] + j0, nullptr, nullptr, (uint32_t)jn * 32u, A.err)) return;
    double xi[I][3];
    long long ii[I];
#pragma unroll
    for (int k = 0; k < I; ++k) {
      ii[k] = i0 + k * T + tid;
      double4_32a p = make_double4_32a(0., 0., 0., 0.);
      if (ii[k] < n) p = A.p64[rb][ii[k]];
      xi[k][0] = p.x, xi[k][1] = p.y, xi[k][2] = p.z;
    }
    const long long iend = i0 + T * I;
    for (int g0 = 0; g0 < jn; g0 += kSeg) {
      const int g1 = min(g0 + kSeg, jn);
      const bool diag = (j0 + g0 < iend) && (i0 < j0 + g1);
      if (diag)
        segment_f64<I, true>(sp, g0, g1, j0, xi, ii, acc);
      else
        segment_f64<I, false>(sp, g0, g1, j0, xi, ii, acc);
    }
  }

  pdl_trigger();
  double4_32a* part = reinterpret_cast<double4_32a*>(A.part);
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const long long i = i0 + k * T + tid;
    if (i < n) {
      double2* r = reinterpret_cast<double2*>(part + blockIdx.y * n + i);
      __stcg(r, make_double2(acc[k][0], acc[k][1]));
      __stcg(r + 1, make_double2(acc[k][2], 0.0));
    }
  }
  if (!arrive_last(&A.cnt[blockIdx.x], gridDim.y, &s_flag)) return;

  if (tid == 0) s_cos = force_time_cos(A, ns);
  __syncthreads();
  if (tid < IONTRAP_MAX_SPECIES) trap_springs(A.trap, A.spc[tid], s_cos, s_springs[tid]);
  __syncthreads();
  const int wb = rb ^ 1;
  const int nsplit = gridDim.y;
#pragma unroll
  for (int k = 0; k < I; ++k) {
    const long long i = i0 + k * T + tid;
    if (i >= n) continue;
    double S[3];
    merge_f64(part, n, i, nsplit, S);
    epilogue_ion<true>(A, i, S, s_springs, ns, wb);
  }
  finish_iblock(A, ns);
}

// ------------------------------------------------------------------ helpers
// Write pair stream b from the FP64 positions x_n (create and force evaluation).
__global__ void k_prep(const __grid_constant__ StepArgs A, int b, int f64) {
  const long long n = A.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double xn[3] = {A.x[i], A.x[n + i], A.x[2 * n + i]};
    const float w = A.spc[A.sp[i]].w;
    if (f64)
      write_pair<true>(A, b, i, xn, w);
    else
      write_pair<false>(A, b, i, xn, w);
  }
}

// Write pair stream b from a full state (x_n, v_n, a_n): the drifted positions
// x_{n+1} = x_n + dt (v_n + dt/2 a_n), by the same operations the epilogue uses.
__global__ void k_restore(const __grid_constant__ StepArgs A, int b, int f64) {
  const long long n = A.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double xn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      xn[c] = drift(A.x[c * n + i], half_kick(A.v[c * n + i], A.a[c * n + i], A.trap.hdt), A.trap.dt);
    const float w = A.spc[A.sp[i]].w;
    if (f64)
      write_pair<true>(A, b, i, xn, w);
    else
      write_pair<false>(A, b, i, xn, w);
  }
}

__global__ void k_normals(unsigned long long seed, long long counter, const long long* ids, long long m, int f64,
                          double* z) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= m) return;
  double t[3];
  if (f64) {
    normals3_f64(seed, counter, ids[k], t);
  } else {
    float tf[3];
    normals3_f32(seed, counter, ids[k], tf);
    t[0] = tf[0], t[1] = tf[1], t[2] = tf[2];
  }
  z[k] = t[0];
  z[m + k] = t[1];
  z[2 * m + k] = t[2];
}

// ------------------------------------------------------------------ registry
struct KernelEntry {
  int f64, T, I, packed, fused;
  const void* fn;
};

#define IT_F32(T, I, P) {0, T, I, P, 1, (const void*)k_step_f32<T, I, P, true>}, \
                        {0, T, I, P, 0, (const void*)k_step_f32<T, I, P, false>}, \
                        {0, T, I, P, 2, (const void*)k_step_f32_cl<T, I, P>}
#define IT_CW(I, W, P) {0, 32 * W, I, P, 3, (const void*)k_step_f32_cw<I, W, P>}
static const KernelEntry kKernels[] = {
    IT_CW(1, 2, false), IT_CW(1, 4, false), IT_CW(2, 2, true), IT_CW(2, 4, true),
    IT_F32(32, 1, false),  IT_F32(32, 2, true),
    IT_F32(64, 1, false),  IT_F32(64, 2, false),  IT_F32(64, 2, true),  IT_F32(64, 4, true),
    IT_F32(128, 1, false), IT_F32(128, 2, false), IT_F32(128, 2, true), IT_F32(128, 4, false),
    IT_F32(128, 4, true),  IT_F32(256, 1, false), IT_F32(256, 2, true), IT_F32(256, 4, true),
    IT_F32(256, 4, false),
    {1, 64, 1, 0, 1, (const void*)k_step_f64<64, 1>},   {1, 128, 1, 0, 1, (const void*)k_step_f64<128, 1>},
    {1, 128, 2, 0, 1, (const void*)k_step_f64<128, 2>}, {1, 256, 1, 0, 1, (const void*)k_step_f64<256, 1>},
};
#undef IT_F32
#undef IT_CW

const void* step_kernel(int f64, int T, int I, int packed, int fused) {
  for (const auto& e : kKernels)
    if (e.f64 == f64 && e.T == T && e.I == I && e.packed == packed && e.fused == fused) return e.fn;
  return nullptr;
}

// Form 3 kernels may be launched in clusters of up to 16 CTAs (non-portable size).
cudaError_t allow_large_clusters() {
  for (const auto& e : kKernels)
    if (e.fused == 3) {
      cudaError_t err = cudaFuncSetAttribute(e.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (err != cudaSuccess) return err;
    }
  return cudaSuccess;
}

const void* epilogue_kernel(int f64) { return f64 ? nullptr : (const void*)k_epilogue_f32; }

const void* prep_kernel() { return (const void*)k_prep; }
const void* restore_kernel() { return (const void*)k_restore; }

cudaError_t launch_normals(unsigned long long seed, long long counter, const long long* d_ids, long long m,
                           int f64, double* d_z, cudaStream_t st) {
  const int T = 128;
  const long long blocks = (m + T - 1) / T;
  k_normals<<<(unsigned)blocks, T, 0, st>>>(seed, counter, d_ids, m, f64, d_z);
  return cudaGetLastError();
}

}  // namespace it
