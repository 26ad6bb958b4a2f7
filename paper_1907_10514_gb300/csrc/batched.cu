// batched.cu -- many independent trap simulations advanced by one launch (sm_103a).
//
// Each ensemble (N <= 2048, FP32 form) keeps its positions resident in shared memory and
// its FP64 state in registers for all K steps of a launch, so a step costs no
// global-memory traffic and no kernel boundary.  Two kernels share the work:
//   N <= 256         k_batched: CTAs of 128 threads (4 warps, 2 ions per lane on packed
//                    FP32x2 instructions, 64 ions per warp); an ensemble of <= 64 ions is
//                    one warp (up to four share a CTA), a larger one a whole CTA; the CTA
//                    barrier is the only synchronisation
//   256 < N <= 2048  k_batched_rp: groups of 2, 4 or 8 CTAs of 256 threads inside a
//                    cluster of 8, part-major like the row-persistent form, positions
//                    exchanged through distributed shared memory, one cluster barrier per
//                    step (no spin-wait on memory)
// The two grids run on two streams side by side.  In both, the summation order of an
// ion's Coulomb sum is a function of N only: an ensemble's trajectory is the same bits
// alone or packed with any other ensembles.
//
// k_batched: the Coulomb sum of an ion runs over j ascending in 64-ion chunks (plain FP32
// inside a chunk, Kahan across chunks).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "iontrap_internal.cuh"

namespace cg = cooperative_groups;

namespace it {

// tuning table of the batched launch (iontrap_api.cu)
bool batched_tuned_shape(int dev, long long n, int* C, int* NP);

constexpr int kBThreads = 128;
constexpr int kBWarps = kBThreads / 32;
constexpr int kBWarpIons = 64;
constexpr int kBCtaIons = kBWarps * kBWarpIons;  // 256
constexpr int kBMaxN = 2048;                     // largest batched ensemble
constexpr int kBChunk = 64;


struct BatchCta {
  int nens;         // ensembles whose stream this CTA holds (0 = idle CTA)
  int ens[kBWarps];
  int soff[kBWarps];       // float4 offset of each ensemble's hi block in shared memory
  int warp_le[kBWarps];    // local ensemble index served by each warp, -1 idle
  int warp_i0[kBWarps];    // first ion of each warp's 64-ion slice
};

// Every CTA holds whole ensembles and only syncs itself.
__global__ void __launch_bounds__(kBThreads)
    k_batched(BatchEns* __restrict__ E, const BatchCta* __restrict__ J, int K) {
  extern __shared__ __align__(16) float4 sm[];
  __shared__ BatchCta job;
  __shared__ double s_springs[kBWarps][IONTRAP_MAX_SPECIES][3];
  __shared__ int s_steps[kBWarps];
  __shared__ long long s_n0[kBWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) job = J[blockIdx.x];
  __syncthreads();
  if (tid < job.nens) {
    const BatchEns& e = E[job.ens[tid]];
    s_steps[tid] = (int)min((long long)K, e.remaining);
    s_n0[tid] = *e.step;
  }
  __syncthreads();
  // stage each held ensemble's pair stream (positions x_{n+1}) into shared memory
  for (int le = 0; le < job.nens; ++le) {
    const BatchEns& e = E[job.ens[le]];
    const int n = (int)e.n;
    const int b = (int)((s_n0[le] + 1) & 1);
    for (int k = tid; k < n; k += kBThreads) {
      sm[job.soff[le] + k] = e.hi[b][k];
      sm[job.soff[le] + n + k] = e.lo[b][k];
    }
  }
  // this warp's two ions and their FP64 state
  const int le = job.warp_le[warp];
  const BatchEns* ens = le >= 0 ? &E[job.ens[le]] : nullptr;
  const int n = ens ? (int)ens->n : 0;
  const int ii[2] = {job.warp_i0[warp] + lane, job.warp_i0[warp] + 32 + lane};
  double x[2][3], v[2][3], a[2][3];
  int spi[2] = {0, 0};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const bool ok = ens && ii[q] < n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[q][c] = ok ? ens->x[c * n + ii[q]] : 0.0;
      v[q][c] = ok ? ens->v[c * n + ii[q]] : 0.0;
      a[q][c] = ok ? ens->a[c * n + ii[q]] : 0.0;
    }
    spi[q] = ok ? ens->sp[ii[q]] : 0;
  }
  bool finite = true;
  // drift and half kick toward the next force evaluation; afterwards they are carried
  // from step to step (the next step's values are the ones each step ends with)
  double xf[2][3], vd[2][3];
  if (ens) {
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vd[q][c] = half_kick(v[q][c], a[q][c], ens->trap.hdt);
        xf[q][c] = drift(x[q][c], vd[q][c], ens->trap.dt);
      }
  }
  __syncthreads();  // every stream staged

  // the ensembles of one CTA may have different step counts: the loop runs to K
  for (int k = 0; k < K; ++k) {
    // per held ensemble: RF phase at the force time, then its species' spring constants
    if (tid < job.nens && k < s_steps[tid]) {
      const BatchEns& e = E[job.ens[tid]];
      const TrapDev& tp = e.trap;
      const long long nf = s_n0[tid] + k + 1;
      const double cosv =
          (tp.flags & (IONTRAP_RF_OFF | IONTRAP_TRAP_OFF | IONTRAP_PSEUDO)) ? 0.0 : cos(tp.Omega * ((double)nf * tp.dt));
      for (int sp = 0; sp < e.nspecies; ++sp) trap_springs(tp, e.spc[sp], cosv, s_springs[tid][sp]);
    }
    __syncthreads();
    const bool active = ens && k < s_steps[le];
    // the force-independent part of the acceleration, ahead of the pair loop
    double ext[2][3];
    if (active) {
      const long long ns = s_n0[le] + k;
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (ii[q] < n) accel_ext<false>(ens->trap, ens->spc[spi[q]], s_springs[le][spi[q]], xf[q], vd[q], ns + 1, ii[q], ext[q]);
    }
    double S[2][3];
    if (active) {
      const float4* sh = sm + job.soff[le];
      const float4* sl = sh + n;
      float2 nxh[1][3], nxl[1][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 h0 = ii[0] < n ? sh[ii[0]] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 h1 = ii[1] < n ? sh[ii[1]] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 l0 = ii[0] < n ? sl[ii[0]] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 l1 = ii[1] < n ? sl[ii[1]] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float hh0 = c == 0 ? h0.x : (c == 1 ? h0.y : h0.z), hh1 = c == 0 ? h1.x : (c == 1 ? h1.y : h1.z);
        const float ll0 = c == 0 ? l0.x : (c == 1 ? l0.y : l0.z), ll1 = c == 0 ? l1.x : (c == 1 ? l1.y : l1.z);
        nxh[0][c] = make_float2(-hh0, -hh1);
        nxl[0][c] = make_float2(-ll0, -ll1);
      }
      const long long iil[2] = {ii[0], ii[1]};
      float ks[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, kc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
      const int w0 = job.warp_i0[warp];
      for (int j0 = 0; j0 < n; j0 += kBChunk) {
        const int jn = min(kBChunk, n - j0);
        float2 acc[1][3] = {{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)}};
        if (ens->unitw) {
          if (j0 == w0)
            segment_f32x2<2, true, true>(sh + j0, sl + j0, jn, j0, nxh, nxl, iil, acc);
          else
            segment_f32x2<2, false, true>(sh + j0, sl + j0, jn, j0, nxh, nxl, iil, acc);
        } else {
          if (j0 == w0)
            segment_f32x2<2, true>(sh + j0, sl + j0, jn, j0, nxh, nxl, iil, acc);
          else
            segment_f32x2<2, false>(sh + j0, sl + j0, jn, j0, nxh, nxl, iil, acc);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float av[2] = {acc[0][c].x, acc[0][c].y};
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const float y = av[q] - kc[q][c];
            const float t = ks[q][c] + y;
            kc[q][c] = (t - ks[q][c]) - y;
            ks[q][c] = t;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) S[q][c] = (double)kc[q][c] - (double)ks[q][c];  // negated sums
    }
    __syncthreads();  // every read of the stream is done
    if (active) {
      const TrapDev& tp = ens->trap;
      float4* sh = sm + job.soff[le];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (ii[q] >= n) continue;
        const SpeciesDev& sd = ens->spc[spi[q]];
        double acc[3], xn[3];
        accel_total(sd, S[q], ext[q], acc);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double vn = half_kick(vd[q][c], acc[c], tp.hdt);
          const double vh = half_kick(vn, acc[c], tp.hdt);
          xn[c] = drift(xf[q][c], vh, tp.dt);
          finite = finite && isfinite(acc[c]) && isfinite(vn) && isfinite(xn[c]);
          x[q][c] = xf[q][c];
          v[q][c] = vn;
          a[q][c] = acc[c];
          xf[q][c] = xn[c];
          vd[q][c] = vh;
        }
        float hv[3], lv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          hv[c] = __double2float_rn(xn[c]);
          lv[c] = __double2float_rn(xn[c] - (double)hv[c]);
        }
        const float4 h4 = make_float4(hv[0], hv[1], hv[2], sd.w);
        const float4 l4 = make_float4(lv[0], lv[1], lv[2], 0.0f);
        sh[ii[q]] = h4;
        sh[n + ii[q]] = l4;
      }
    }
    __syncthreads();  // new entries visible
  }

  // write back: FP64 state, the pair stream x_{n+1} of the final state, step, flags
  if (ens) {
    const int steps = s_steps[le];
    const long long nend = s_n0[le] + steps;
    const int b = (int)((nend + 1) & 1);
    const float4* sh = sm + job.soff[le];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (ii[q] >= n) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        ens->x[c * n + ii[q]] = x[q][c];
        ens->v[c * n + ii[q]] = v[q][c];
        ens->a[c * n + ii[q]] = a[q][c];
      }
      ens->hi[b][ii[q]] = sh[ii[q]];
      ens->lo[b][ii[q]] = sh[n + ii[q]];
    }
    if (!finite) atomicOr(ens->err, ERR_NONFINITE);
    if (job.warp_i0[warp] == 0 && lane == 0) {  // one thread per ensemble
      *ens->step = nend;
      E[job.ens[le]].remaining -= steps;
    }
  }
}

// ------------------------------------------------------------------ part-major groups
// Ensembles of 257..2048 ions: a group of C = 2, 4 or 8 CTAs of kBRThreads threads inside a
// cluster of kBRCluster CTAs, each CTA owning R = ceil(n / C) ions.  Every CTA holds the whole ensemble as part-major SoA floats (NP parts of JP
// entries: x_hi, y_hi, z_hi, x_lo, y_lo, z_lo) in two shared-memory buffers, the positions
// of the current step and those of the next, which the owners of every CTA of the group
// write through distributed shared memory, and the charges z once.  The pair work is R x NP items (ion slot s, part p), item
// m = p R + s, taken round-robin by the threads (NP chosen so that the threads are busy in
// every round); the part partials merge in part order and thread s < R integrates ion
// r R + s in FP64.  One cluster barrier per step.
//
// Summation order: per part, j ascending in 128-j chunks (even and odd j summed apart and
// added), chunks Kahan-added, parts Kahan-merged in order -- a function of n only (C, R,
// NP and JP are), so an ensemble's trajectory is the same bits alone or in any mix.
constexpr int kBRThreads = 256;
constexpr int kBRCluster = 8;
constexpr int kBRMaxParts = 16;

struct BatchRpCta {
  int e;      // ensemble, -1: idle CTA
  int r;      // this CTA's index in the ensemble's group
  int rank0;  // cluster rank of the group's first CTA
  int C;      // CTAs in the group
  int R;      // ions per CTA: ceil(n / C)
  int NP;     // j-parts
  int JP;     // entries per part: a multiple of 4 (JP / 4 odd when R % 32 != 0)
};

// Shared memory of a group CTA: two buffers of NP x 6 x JP floats, the charges (NP x JP)
// and the part partials (sum, compensation) [NP][3][R] floats each.  At most ~113 KB (two
// CTAs per SM) up to n ~ 2048.
static size_t brp_smem_bytes(int R, int NP, int JP) {
  return 13 * (size_t)NP * JP * sizeof(float) + 2 * (size_t)NP * 3 * R * sizeof(float);
}

__global__ void __launch_bounds__(kBRThreads, 2)
    k_batched_rp(BatchEns* __restrict__ E, const BatchRpCta* __restrict__ J, int K) {
  extern __shared__ __align__(16) float4 sm[];
  __shared__ double s_springs[IONTRAP_MAX_SPECIES][3];
  __shared__ int s_next;  // the step's next (ion, part) item past the first round
  const int tid = threadIdx.x;
  const BatchRpCta job = J[blockIdx.x];
  BatchEns* ens = job.e >= 0 ? E + job.e : nullptr;
  const int n = ens ? (int)ens->n : 0;
  const int R = job.R, NP = job.NP, JP = job.JP;
  const int blen = NP * 6 * JP;  // floats per buffer
  float* buf = reinterpret_cast<float*>(sm);
  float* wz = buf + 2 * blen;     // charges, [NP][JP]
  float* ps = wz + NP * JP;
  float* pc = ps + NP * 3 * R;
  // read before the first barrier; the group's first CTA rewrites them after the last
  const int steps = ens ? (int)min((long long)K, ens->remaining) : 0;
  const long long n0 = ens ? *ens->step : 0;
  cg::cluster_group cluster = cg::this_cluster();

  // stage the positions x_{n0+1} into buffer 0, the padding into both buffers and the
  // charges (padding entries sit at 1e30 m: r^2 overflows, rsqrt gives 0, the term is 0)
  if (steps > 0) {
    const int b = (int)((n0 + 1) & 1);
    const float4* __restrict__ gh = ens->hi[b];
    const float4* __restrict__ gl = ens->lo[b];
    for (int e = tid; e < NP * JP; e += kBRThreads) {
      const int p = e / JP, q = e - p * JP;
      float4 h = make_float4(1e30f, 1e30f, 1e30f, 0.f), l = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < n) {
        h = gh[e];
        l = gl[e];
      }
      float* d = buf + p * 6 * JP + q;
      d[0] = h.x, d[JP] = h.y, d[2 * JP] = h.z;
      d[3 * JP] = l.x, d[4 * JP] = l.y, d[5 * JP] = l.z;
      wz[e] = h.w;
      float* d1 = d + blen;
      if (e >= n) {
        d1[0] = d1[JP] = d1[2 * JP] = 1e30f;
        d1[3 * JP] = d1[4 * JP] = d1[5 * JP] = 0.f;
      }
    }
  }
  // the owned ion and its FP64 state: drift and half kick toward the next force
  // evaluation, carried from step to step
  const int r0 = job.r * R;
  const int Rg = steps > 0 ? max(0, min(R, n - r0)) : 0;
  const bool own = tid < Rg;
  const int ie = r0 + tid;
  const int eo = own ? (ie / JP) * 6 * JP + (ie % JP) : 0;  // ion ie's entry in a buffer
  int spi = 0;
  double xf[3] = {0.0, 0.0, 0.0}, vd[3] = {0.0, 0.0, 0.0};
  if (own) {
    spi = ens->sp[ie];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      vd[c] = half_kick(ens->v[c * n + ie], ens->a[c * n + ie], ens->trap.hdt);
      xf[c] = drift(ens->x[c * n + ie], vd[c], ens->trap.dt);
    }
  }
  bool finite = true;
  cluster.sync();  // every copy staged before the first remote write

  int cur = 0;
  for (int k = 0; k < K; ++k) {
    const bool active = k < steps;
    if (active && tid < ens->nspecies) {  // this step's spring constants per species
      const TrapDev& tp = ens->trap;
      const double cosv = (tp.flags & (IONTRAP_RF_OFF | IONTRAP_TRAP_OFF | IONTRAP_PSEUDO))
                              ? 0.0
                              : cos(tp.Omega * ((double)(n0 + k + 1) * tp.dt));
      trap_springs(tp, ens->spc[tid], cosv, s_springs[tid]);
    }
    if (tid == 0) s_next = kBRThreads;
    __syncthreads();
    // the force-independent part of the acceleration, ahead of the pair work
    double ext[3];
    if (own && active) accel_ext<false>(ens->trap, ens->spc[spi], s_springs[spi], xf, vd, n0 + k + 1, ie, ext);
    if (active) {
      const float* sb = buf + cur * blen;
      const bool unitw = ens->unitw != 0;
      // the first round of items by thread index, the rest to whichever thread is free
      // (the owners start late: they evaluate the trap, drag and noise first); each item's
      // sum is its own, so the bits do not depend on which thread takes it
      for (int m = tid; m < R * NP; m = atomicAdd(&s_next, 1)) {
        const int p = m / R, s = m - p * R;
        const int i = r0 + s;
        if (i >= n) continue;
        const float* si = sb + (i / JP) * 6 * JP + (i % JP);
        const float2 nh[3] = {make_float2(-si[0], -si[0]), make_float2(-si[JP], -si[JP]),
                              make_float2(-si[2 * JP], -si[2 * JP])};
        const float2 nl[3] = {make_float2(-si[3 * JP], -si[3 * JP]), make_float2(-si[4 * JP], -si[4 * JP]),
                              make_float2(-si[5 * JP], -si[5 * JP])};
        const float* sj = sb + p * 6 * JP;
        const float* sw = wz + p * JP;
        float ks[3] = {0.f, 0.f, 0.f}, kcp[3] = {0.f, 0.f, 0.f};
        for (int c0 = 0; c0 < JP; c0 += kSeg) {
          const int qn = min(kSeg, JP - c0);
          float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          // the self pair can only sit in a chunk that overlaps the CTA's own ions; the
          // variant is chosen per warp (its lanes may hold different items)
          const int jc = p * JP + c0;
          const bool diag = __any_sync(__activemask(), (jc < r0 + Rg) && (r0 < jc + qn));
          if (unitw) {
            if (diag)
              rp_chunk<true, true>(sj + c0, sw + c0, JP, qn, jc, i, nh, nl, acc);
            else
              rp_chunk<false, true>(sj + c0, sw + c0, JP, qn, jc, i, nh, nl, acc);
          } else {
            if (diag)
              rp_chunk<true, false>(sj + c0, sw + c0, JP, qn, jc, i, nh, nl, acc);
            else
              rp_chunk<false, false>(sj + c0, sw + c0, JP, qn, jc, i, nh, nl, acc);
          }
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float a = acc[d].x + acc[d].y;
            const float y = a - kcp[d];
            const float t = ks[d] + y;
            kcp[d] = (t - ks[d]) - y;
            ks[d] = t;
          }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          ps[(p * 3 + d) * R + s] = ks[d];
          pc[(p * 3 + d) * R + s] = kcp[d];
        }
      }
    }
    __syncthreads();
    if (own && active) {  // merge in part order (Kahan), integrate, publish the next positions
      double S[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float su = 0.f, cu = 0.f;
        for (int p = 0; p < NP; ++p) kahan_merge(su, cu, ps[(p * 3 + d) * R + tid], pc[(p * 3 + d) * R + tid]);
        S[d] = (double)cu - (double)su;  // the accumulators hold the negated sum
      }
      const SpeciesDev& sd = ens->spc[spi];
      const TrapDev& tp = ens->trap;
      double acc[3];
      accel_total(sd, S, ext, acc);
      const bool last = k == steps - 1;
      float h[3], l[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double vn = half_kick(vd[c], acc[c], tp.hdt);
        const double vh = half_kick(vn, acc[c], tp.hdt);
        const double xn = drift(xf[c], vh, tp.dt);
        finite = finite && isfinite(acc[c]) && isfinite(vn) && isfinite(xn);
        if (last) {
          ens->x[c * n + ie] = xf[c];
          ens->v[c * n + ie] = vn;
          ens->a[c * n + ie] = acc[c];
        }
        xf[c] = xn;
        vd[c] = vh;
        h[c] = __double2float_rn(xn);
        l[c] = __double2float_rn(xn - (double)h[c]);
      }
      float* dl = buf + (cur ^ 1) * blen + eo;
      for (int rr = 0; rr < job.C; ++rr) {
        float* d = cluster.map_shared_rank(dl, (unsigned)(job.rank0 + rr));
        d[0] = h[0], d[JP] = h[1], d[2 * JP] = h[2];
        d[3 * JP] = l[0], d[4 * JP] = l[1], d[5 * JP] = l[2];
      }
      if (last) {  // the pair stream of the final state, x_{n+1}
        const int bn = (int)((n0 + steps + 1) & 1);
        ens->hi[bn][ie] = make_float4(h[0], h[1], h[2], sd.w);
        ens->lo[bn][ie] = make_float4(l[0], l[1], l[2], 0.f);
      }
    }
    cluster.sync();  // every CTA's reads of this step's buffer and writes of the next are done
    cur ^= 1;
  }
  if (own && !finite) atomicOr(ens->err, ERR_NONFINITE);
  if (steps > 0 && job.r == 0 && tid == 0) {  // one thread per ensemble
    *ens->step = n0 + steps;
    ens->remaining -= steps;
  }
}

// ------------------------------------------------------------------ host side
struct BatchPlan {
  std::vector<BatchRpCta> groups;   // part-major groups of 2, 4 or 8 CTAs (clusters of 8)
  std::vector<BatchCta> single;     // CTAs holding whole ensembles of <= 256 ions (no cluster)
  size_t smem_groups = 0, smem_single = 0;
};

// Part count of a part-major CTA with R ions of an n-ion ensemble: the threads take the
// R x NP items in ceil(R NP / threads) rounds of JP entries each, so NP minimises
// rounds x (JP + the per-item overhead in pair equivalents), within the shared memory
// that lets two CTAs share an SM if any shape fits there, else within the CTA limit.
constexpr int kBRItemCost = 8;
constexpr size_t kBRSmemTwo = 112 * 1024;  // two CTAs per SM (228 KB less 1 KB each reserved, static arrays)
constexpr size_t kBRSmemOne = 226 * 1024;  // 227 KB less the static arrays
static int brp_jp(int n, int R, int np) {
  long long q4 = ((n + np - 1) / np + 3) / 4;
  if (R % 32 != 0 && !(q4 & 1)) ++q4;
  return (int)(4 * q4);
}

static void brp_shape(int n, int C, int np_tuned, BatchRpCta* t) {
  const int R = (n + C - 1) / C;
  t->R = R;
  t->C = C;
  // a part count from the tuning table, if it fits in a CTA's shared memory
  if (np_tuned > 0 && np_tuned <= kBRMaxParts && brp_smem_bytes(R, np_tuned, brp_jp(n, R, np_tuned)) <= kBRSmemOne) {
    t->NP = np_tuned;
    t->JP = brp_jp(n, R, np_tuned);
    return;
  }
  for (size_t lim : {kBRSmemTwo, kBRSmemOne}) {
    long long best = -1;
    for (int np = 1; np <= kBRMaxParts; ++np) {
      long long q4 = ((n + np - 1) / np + 3) / 4;
      if (R % 32 != 0 && !(q4 & 1)) ++q4;
      const int jp = (int)(4 * q4);
      if (brp_smem_bytes(R, np, jp) > lim) continue;
      const long long rounds = ((long long)R * np + kBRThreads - 1) / kBRThreads;
      const long long cost = rounds * (jp + kBRItemCost);
      if (best < 0 || cost < best) {
        best = cost;
        t->NP = np;
        t->JP = jp;
      }
    }
    if (best >= 0) break;
  }
}

// Group shape of the part-major groups for an ensemble of n ions (256 < n <= 2048): the
// CTAs per group C and the j-part count NP (0: the cost model of brp_shape) from the
// tuning table of device dev (iontrap_autotune_many), else 2 CTAs up to 512 ions, 4 up to
// 1024, 8 above.  A function of (dev, n) and the table only.
static void brp_group(int dev, long long n, int* C, int* NP) {
  *C = n <= 512 ? 2 : (n <= 1024 ? 4 : 8);
  *NP = 0;
  int tc = 0, tnp = 0;
  if (batched_tuned_shape(dev, n, &tc, &tnp) && (tc == 2 || tc == 4 || tc == 8) && (n + tc - 1) / tc <= kBRThreads) {
    *C = tc;
    *NP = tnp;
  }
}

// Pack ensembles (sizes n[e]) into CTAs.  Above 256 ions: part-major groups of C CTAs
// (brp_group), placed buddy-aligned in clusters of 8 (largest first, similar sizes
// together).  The rest one per CTA (64 < N <= 256) or four per CTA (N <= 64), heaviest
// first, in a grid without clusters.
static BatchPlan plan_batch(const std::vector<long long>& n, int dev) {
  BatchPlan plan;
  struct Job {
    int e;
    int ctas;
    long long work;
    int np;
  };
  std::vector<Job> big, mid, small;
  for (int e = 0; e < (int)n.size(); ++e) {
    if (n[e] <= kBWarpIons) {
      small.push_back({e, 1, n[e] * n[e], 0});
    } else if (n[e] <= kBCtaIons) {
      mid.push_back({e, 1, n[e] * n[e], 0});
    } else {
      int C = 0, NP = 0;
      brp_group(dev, n[e], &C, &NP);
      big.push_back({e, C, n[e] * n[e], NP});
    }
  }
  auto heavier = [](const Job& a, const Job& b) { return a.ctas != b.ctas ? a.ctas > b.ctas : a.work > b.work; };
  std::sort(big.begin(), big.end(), heavier);
  std::sort(mid.begin(), mid.end(), heavier);
  std::sort(small.begin(), small.end(), heavier);
  auto blank = []() {
    BatchCta c{};
    c.nens = 0;
    for (int w = 0; w < kBWarps; ++w) c.warp_le[w] = -1;
    return c;
  };
  auto whole = [&](const Job& j) {
    BatchCta t = blank();
    t.nens = 1;
    t.ens[0] = j.e;
    t.soff[0] = 0;
    for (int w = 0; w < kBWarps; ++w) {
      const long long i0 = (long long)w * kBWarpIons;
      if (i0 < n[j.e]) {
        t.warp_le[w] = 0;
        t.warp_i0[w] = (int)i0;
      }
    }
    return t;
  };
  // part-major groups: buddy placement of the groups of 2, 4 and 8 inside clusters of 8
  int used = 0;
  for (const Job& j : big) {
    BatchRpCta t{};
    t.e = j.e;
    brp_shape((int)n[j.e], j.ctas, j.np, &t);
    const size_t smem = brp_smem_bytes(t.R, t.NP, t.JP);
    while (used % j.ctas) {
      BatchRpCta idle{};
      idle.e = -1;
      plan.groups.push_back(idle);
      ++used;
    }
    if (used == kBRCluster) used = 0;
    t.rank0 = used;
    for (int r = 0; r < j.ctas; ++r) {
      t.r = r;
      plan.groups.push_back(t);
    }
    used += j.ctas;
    if (used == kBRCluster) used = 0;
    plan.smem_groups = std::max(plan.smem_groups, smem);
  }
  while (plan.groups.size() % kBRCluster) {
    BatchRpCta idle{};
    idle.e = -1;
    plan.groups.push_back(idle);
  }
  // single grid
  for (const Job& j : mid) {
    plan.single.push_back(whole(j));
    plan.smem_single = std::max(plan.smem_single, (size_t)n[j.e] * 2 * sizeof(float4));
  }
  for (size_t k = 0; k < small.size(); k += kBWarps) {
    BatchCta t = blank();
    int off = 0;
    for (int w = 0; w < kBWarps && k + w < small.size(); ++w) {
      const int e = small[k + w].e;
      t.ens[w] = e;
      t.soff[w] = off;
      t.warp_le[w] = w;
      t.warp_i0[w] = 0;
      off += (int)n[e] * 2;
      t.nens = w + 1;
    }
    plan.single.push_back(t);
    plan.smem_single = std::max(plan.smem_single, (size_t)off * sizeof(float4));
  }
  return plan;
}

// Device buffers of the batched launcher, grown on demand: one set per (device, calling
// stream), so that batched launches on different streams run side by side.
struct BatchBuffers {
  BatchEns* d_ens = nullptr;
  size_t ens_cap = 0;
  BatchCta* d_cta = nullptr;
  size_t cta_cap = 0;
  BatchRpCta* d_rp = nullptr;
  size_t rp_cap = 0;
  cudaStream_t side = nullptr;  // second stream: the small-ensemble grid runs beside the clustered one
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t done = nullptr;   // recorded after the previous launches, which read the tables
  bool pending = false;
  std::mutex mu;                // one call at a time uses a set
  int dev = -1;                 // owner of the set: (device, stream), and when it was last used
  cudaStream_t stream = nullptr;
  unsigned long long used = 0;
};
// At most kBatchSets sets; a stream without one takes the least recently used set, which
// first waits for the launches that read its tables (and gets a side stream of the new
// stream's priority).
constexpr int kBatchSets = 16;
static std::mutex g_bb_mu;
static BatchBuffers g_bbs[kBatchSets];
static unsigned long long g_bb_clock = 0;

static BatchBuffers& buffers_for(int dev, cudaStream_t stream) {
  std::lock_guard<std::mutex> lock(g_bb_mu);
  BatchBuffers* pick = nullptr;
  for (BatchBuffers& b : g_bbs)
    if (b.dev == dev && b.stream == stream) pick = &b;
  if (!pick) {
    pick = &g_bbs[0];
    for (BatchBuffers& b : g_bbs)
      if (b.used < pick->used) pick = &b;
    std::lock_guard<std::mutex> set_lock(pick->mu);
    if (pick->pending) cudaEventSynchronize(pick->done);
    pick->pending = false;
    if (pick->dev != dev && pick->done) {  // buffers of another device: start afresh on this one
      int cur = -1;
      cudaGetDevice(&cur);
      cudaSetDevice(pick->dev);
      cudaFree(pick->d_ens), cudaFree(pick->d_cta), cudaFree(pick->d_rp);
      cudaStreamDestroy(pick->side);
      cudaEventDestroy(pick->fork), cudaEventDestroy(pick->join), cudaEventDestroy(pick->done);
      cudaSetDevice(cur);
      pick->d_ens = nullptr, pick->d_cta = nullptr, pick->d_rp = nullptr;
      pick->ens_cap = pick->cta_cap = pick->rp_cap = 0;
      pick->side = nullptr, pick->fork = pick->join = pick->done = nullptr;
    } else if (pick->side) {  // same device: the side stream takes the new stream's priority
      cudaStreamDestroy(pick->side);
      int prio = 0;
      if (stream) cudaStreamGetPriority(stream, &prio);
      if (cudaStreamCreateWithPriority(&pick->side, cudaStreamNonBlocking, prio) != cudaSuccess) pick->side = nullptr;
    }
    pick->dev = dev;
    pick->stream = stream;
  }
  pick->used = ++g_bb_clock;
  return *pick;
}

int batched_max_n() { return kBMaxN; }

// Whether a part-major group of C CTAs with NP j-parts (0: the cost model) can hold an
// ensemble of n ions.
bool batched_shape_fits(long long n, int C, int NP) {
  if (n <= kBCtaIons || n > kBMaxN || !(C == 2 || C == 4 || C == 8) || (n + C - 1) / C > kBRThreads) return false;
  if (NP == 0) return true;
  const int R = (int)((n + C - 1) / C);
  return NP > 0 && NP <= kBRMaxParts && brp_smem_bytes(R, NP, brp_jp((int)n, R, NP)) <= kBRSmemOne;
}

static cudaError_t grow(void** p, size_t* cap, size_t need, size_t elem) {
  if (need <= *cap) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const size_t c = std::max(need, (size_t)64);
  cudaError_t e = cudaMalloc(p, c * elem);
  if (e == cudaSuccess) *cap = c;
  return e;
}

// Enqueue `steps[e]` steps of every ensemble on `stream`, K steps per launch.
cudaError_t launch_batched(const std::vector<BatchEns>& ens_in, const std::vector<long long>& steps, int K,
                           cudaStream_t stream) {
  if (ens_in.empty()) return cudaSuccess;
  std::vector<long long> n(ens_in.size());
  long long max_steps = 0;
  for (size_t e = 0; e < ens_in.size(); ++e) {
    n[e] = ens_in[e].n;
    max_steps = std::max(max_steps, steps[e]);
  }
  if (max_steps == 0) return cudaSuccess;
  int dev = 0;
  cudaError_t derr = cudaGetDevice(&dev);
  if (derr != cudaSuccess) return derr;
  BatchPlan plan = plan_batch(n, dev);
  BatchBuffers& g_bb = buffers_for(dev, stream);
  std::lock_guard<std::mutex> set_lock(g_bb.mu);
  cudaError_t err = cudaSuccess;
  if (!g_bb.done) {
    err = cudaEventCreateWithFlags(&g_bb.done, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&g_bb.fork, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&g_bb.join, cudaEventDisableTiming);
    if (err != cudaSuccess) return err;
  }
  if (!g_bb.side) {  // the side stream runs at the calling stream's priority
    int prio = 0;
    if (stream) cudaStreamGetPriority(stream, &prio);
    err = cudaStreamCreateWithPriority(&g_bb.side, cudaStreamNonBlocking, prio);
    if (err != cudaSuccess) return err;
  }
  // The tables of this stream are shared by its calls: wait until the previous launches
  // have finished reading them.
  if (g_bb.pending) {
    err = cudaEventSynchronize(g_bb.done);
    if (err != cudaSuccess) return err;
    g_bb.pending = false;
  }
  const size_t ng = plan.groups.size(), ns = plan.single.size();
  err = grow((void**)&g_bb.d_ens, &g_bb.ens_cap, ens_in.size(), sizeof(BatchEns));
  if (err == cudaSuccess) err = grow((void**)&g_bb.d_cta, &g_bb.cta_cap, ns, sizeof(BatchCta));
  if (err == cudaSuccess) err = grow((void**)&g_bb.d_rp, &g_bb.rp_cap, ng, sizeof(BatchRpCta));
  if (err != cudaSuccess) return err;
  std::vector<BatchEns> ens = ens_in;
  for (size_t e = 0; e < ens.size(); ++e) ens[e].remaining = steps[e];
  // synchronous copies: the host vectors die with this call
  err = cudaStreamSynchronize(stream);
  if (err == cudaSuccess)
    err = cudaMemcpy(g_bb.d_ens, ens.data(), ens.size() * sizeof(BatchEns), cudaMemcpyHostToDevice);
  if (err == cudaSuccess && ns)
    err = cudaMemcpy(g_bb.d_cta, plan.single.data(), ns * sizeof(BatchCta), cudaMemcpyHostToDevice);
  if (err == cudaSuccess && ng)
    err = cudaMemcpy(g_bb.d_rp, plan.groups.data(), ng * sizeof(BatchRpCta), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return err;
  if (ns) err = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(plan.smem_single, 16));
  if (err == cudaSuccess && ng)
    err = cudaFuncSetAttribute(k_batched_rp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem_groups);
  if (err != cudaSuccess) return err;
  // fork: the small-ensemble grid on the side stream, the clustered grid on `stream`
  err = cudaEventRecord(g_bb.fork, stream);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(g_bb.side, g_bb.fork, 0);
  // each grid loops over no more steps per launch than its longest ensemble still needs
  long long max_g = 0, max_s = 0;
  for (const BatchRpCta& t : plan.groups)
    if (t.e >= 0) max_g = std::max(max_g, steps[t.e]);
  for (const BatchCta& t : plan.single)
    for (int w = 0; w < t.nens; ++w) max_s = std::max(max_s, steps[t.ens[w]]);
  for (long long done = 0; done < max_steps && err == cudaSuccess; done += K) {
    const int Kg = (int)std::max<long long>(0, std::min<long long>(K, max_g - done));
    const int Ks = (int)std::max<long long>(0, std::min<long long>(K, max_s - done));
    if (ng && Kg > 0) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3((unsigned)ng);
      cfg.blockDim = dim3(kBRThreads);
      cfg.dynamicSmemBytes = plan.smem_groups;
      cfg.stream = stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = kBRCluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      err = cudaLaunchKernelEx(&cfg, k_batched_rp, g_bb.d_ens, (const BatchRpCta*)g_bb.d_rp, Kg);
    }
    if (ns && Ks > 0 && err == cudaSuccess) {
      k_batched<<<(unsigned)ns, kBThreads, std::max<size_t>(plan.smem_single, 16), g_bb.side>>>(
          g_bb.d_ens, g_bb.d_cta, Ks);
      err = cudaGetLastError();
    }
  }
  // join
  if (err == cudaSuccess) err = cudaEventRecord(g_bb.join, g_bb.side);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(stream, g_bb.join, 0);
  if (err == cudaSuccess) err = cudaEventRecord(g_bb.done, stream);
  if (err == cudaSuccess) g_bb.pending = true;
  return err;
}

}  // namespace it
