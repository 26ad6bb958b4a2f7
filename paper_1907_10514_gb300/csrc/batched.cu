// batched.cu -- many independent trap simulations advanced by one launch (sm_103a).
//
// Each ensemble (N <= 2048, FP32 form) keeps its FP32 hi/lo pair stream resident in
// shared memory and its FP64 state (x, v, a) in registers for all K steps of a launch,
// so a step costs no global-memory traffic and no kernel boundary.  CTAs of 128 threads
// (4 warps, 2 ions per lane on packed FP32x2 instructions, 64 ions per warp) are grouped
// in clusters of 8:
//   N <= 64          one warp; up to four such ensembles share a CTA
//   64 < N <= 256    one CTA
//   256 < N <= 2048  2, 4 or 8 CTAs of one cluster, 256 ions each; every CTA keeps a full
//                    copy of the ensemble's pair stream and writes its ions' new entries
//                    into the other copies through distributed shared memory
// Every step: pair sum over the ensemble's stream -> cluster barrier (all reads done) ->
// integrate own ions, write new stream entries locally and remotely -> cluster barrier.
// The barriers are the hardware cluster barrier: no spin-wait on memory.
//
// The Coulomb sum of an ion runs over j ascending in 64-ion chunks (plain FP32 inside a
// chunk, Kahan across chunks), a function of N only: an ensemble's trajectory is the
// same bits alone or packed with any other ensembles.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "iontrap_internal.cuh"

namespace cg = cooperative_groups;

namespace it {

constexpr int kBCluster = 8;
constexpr int kBThreads = 128;
constexpr int kBWarps = kBThreads / 32;
constexpr int kBWarpIons = 64;
constexpr int kBCtaIons = kBWarps * kBWarpIons;  // 256
constexpr int kBMaxN = kBCluster * kBCtaIons;    // 2048
constexpr int kBChunk = 64;


struct BatchCta {
  int nens;         // ensembles whose stream this CTA holds (0 = idle CTA)
  int ens[kBWarps];
  int soff[kBWarps];       // float4 offset of each ensemble's hi block in shared memory
  int warp_le[kBWarps];    // local ensemble index served by each warp, -1 idle
  int warp_i0[kBWarps];    // first ion of each warp's 64-ion slice
  int rank0, nranks;       // cluster ranks that hold copies of ens[0] (multi-CTA ensemble)
};

// clustered = 1: launched in clusters of 8 (ensembles spread over several CTAs, synced by
// the hardware cluster barrier); 0: every CTA holds whole ensembles and only syncs itself.
__global__ void __launch_bounds__(kBThreads)
    k_batched(BatchEns* __restrict__ E, const BatchCta* __restrict__ J, int K, int clustered) {
  extern __shared__ __align__(16) float4 sm[];
  __shared__ BatchCta job;
  __shared__ double s_springs[kBWarps][IONTRAP_MAX_SPECIES][3];
  __shared__ int s_steps[kBWarps];
  __shared__ long long s_n0[kBWarps];
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned my_rank = clustered ? cluster.block_rank() : 0u;
  auto sync_all = [&]() {
    if (clustered)
      cluster.sync();
    else
      __syncthreads();
  };
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
  sync_all();  // every copy staged before any CTA writes into another's

  // CTAs of one cluster may hold ensembles with different step counts: the loop runs to K
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
    sync_all();  // every read of every stream copy is done
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
        for (int r = job.rank0; r < job.rank0 + job.nranks; ++r) {
          float4* dst = (r == (int)my_rank) ? sh : cluster.map_shared_rank(sh, (unsigned)r);
          dst[ii[q]] = h4;
          dst[n + ii[q]] = l4;
        }
      }
    }
    sync_all();  // new entries visible in every copy
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

// ------------------------------------------------------------------ host side
struct BatchPlan {
  std::vector<BatchCta> clustered;  // CTAs of ensembles spread over 2, 4 or 8 CTAs (clusters of 8)
  std::vector<BatchCta> single;     // CTAs holding whole ensembles (no cluster)
  size_t smem_clustered = 0, smem_single = 0;
};

// Pack ensembles (sizes n[e]) into CTAs: ensembles above one CTA's 256 ions into
// aligned power-of-two groups of clusters of 8 (largest first, similar sizes together);
// the rest one per CTA (64 < N <= 256) or four per CTA (N <= 64), heaviest first, in a
// grid without clusters.
static BatchPlan plan_batch(const std::vector<long long>& n) {
  BatchPlan plan;
  struct Job {
    int e;
    int ctas;
    long long work;
  };
  std::vector<Job> big, mid, small;
  for (int e = 0; e < (int)n.size(); ++e) {
    if (n[e] <= kBWarpIons) {
      small.push_back({e, 1, n[e] * n[e]});
    } else if (n[e] <= kBCtaIons) {
      mid.push_back({e, 1, n[e] * n[e]});
    } else {
      int c = 2;
      while ((long long)c * kBCtaIons < n[e]) c *= 2;
      big.push_back({e, c, n[e] * n[e]});
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
    c.rank0 = 0;
    c.nranks = 1;
    return c;
  };
  auto whole = [&](const Job& j, int r, int r0, int c) {
    BatchCta t = blank();
    t.nens = 1;
    t.ens[0] = j.e;
    t.soff[0] = 0;
    for (int w = 0; w < kBWarps; ++w) {
      const long long i0 = (long long)r * kBCtaIons + (long long)w * kBWarpIons;
      if (i0 < n[j.e]) {
        t.warp_le[w] = 0;
        t.warp_i0[w] = (int)i0;
      }
    }
    t.rank0 = r0;
    t.nranks = c;
    return t;
  };
  // clustered grid: buddy placement of power-of-two groups inside clusters of 8
  int used = 0;
  for (const Job& j : big) {
    while (used % j.ctas) {
      plan.clustered.push_back(blank());
      ++used;
    }
    if (used == kBCluster) used = 0;
    const int r0 = used;
    for (int r = 0; r < j.ctas; ++r) plan.clustered.push_back(whole(j, r, r0, j.ctas));
    used += j.ctas;
    if (used == kBCluster) used = 0;
    plan.smem_clustered = std::max(plan.smem_clustered, (size_t)n[j.e] * 2 * sizeof(float4));
  }
  while (plan.clustered.size() % kBCluster) plan.clustered.push_back(blank());
  // single grid
  for (const Job& j : mid) {
    plan.single.push_back(whole(j, 0, 0, 1));
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

// Device buffers of the batched launcher, grown on demand (one set per process).
struct BatchBuffers {
  BatchEns* d_ens = nullptr;
  size_t ens_cap = 0;
  BatchCta* d_cta = nullptr;
  size_t cta_cap = 0;
  cudaStream_t side = nullptr;  // second stream: the single-CTA grid runs beside the clustered one
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t done = nullptr;   // recorded after the previous launches, which read the tables
  bool pending = false;
};
static BatchBuffers g_bb;

int batched_max_n() { return kBMaxN; }

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
  BatchPlan plan = plan_batch(n);
  cudaError_t err = cudaSuccess;
  if (!g_bb.done) {
    err = cudaEventCreateWithFlags(&g_bb.done, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&g_bb.fork, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&g_bb.join, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&g_bb.side, cudaStreamNonBlocking);
    if (err != cudaSuccess) return err;
  }
  // The tables are shared by all calls: wait until the previous launches, which may run
  // on another (possibly since destroyed) stream, have finished reading them.
  if (g_bb.pending) {
    err = cudaEventSynchronize(g_bb.done);
    if (err != cudaSuccess) return err;
    g_bb.pending = false;
  }
  const size_t nc = plan.clustered.size(), ns = plan.single.size();
  err = grow((void**)&g_bb.d_ens, &g_bb.ens_cap, ens_in.size(), sizeof(BatchEns));
  if (err == cudaSuccess) err = grow((void**)&g_bb.d_cta, &g_bb.cta_cap, nc + ns, sizeof(BatchCta));
  if (err != cudaSuccess) return err;
  std::vector<BatchEns> ens = ens_in;
  for (size_t e = 0; e < ens.size(); ++e) ens[e].remaining = steps[e];
  std::vector<BatchCta> ctas = plan.clustered;
  ctas.insert(ctas.end(), plan.single.begin(), plan.single.end());
  // synchronous copies: the host vectors die with this call
  err = cudaStreamSynchronize(stream);
  if (err == cudaSuccess)
    err = cudaMemcpy(g_bb.d_ens, ens.data(), ens.size() * sizeof(BatchEns), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(g_bb.d_cta, ctas.data(), ctas.size() * sizeof(BatchCta), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return err;
  const size_t smem = std::max<size_t>(std::max(plan.smem_clustered, plan.smem_single), 16);
  err = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  // fork: the single-CTA grid on the side stream, the clustered grid on `stream`
  err = cudaEventRecord(g_bb.fork, stream);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(g_bb.side, g_bb.fork, 0);
  for (long long done = 0; done < max_steps && err == cudaSuccess; done += K) {
    if (nc) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3((unsigned)nc);
      cfg.blockDim = dim3(kBThreads);
      cfg.dynamicSmemBytes = std::max<size_t>(plan.smem_clustered, 16);
      cfg.stream = stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = kBCluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      err = cudaLaunchKernelEx(&cfg, k_batched, g_bb.d_ens, (const BatchCta*)g_bb.d_cta, K, 1);
    }
    if (ns && err == cudaSuccess) {
      k_batched<<<(unsigned)ns, kBThreads, std::max<size_t>(plan.smem_single, 16), g_bb.side>>>(
          g_bb.d_ens, g_bb.d_cta + nc, K, 0);
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
