// persistent.cu -- grid-persistent step form (fused = 4) of libiontrap.so (sm_103a).
//
// One cooperative launch advances a simulation by K velocity-Verlet steps (Sec. 6
// "Integration"); every CTA stays resident for the whole launch.  The work of a step
// is split statically so that every CTA gets the same number of pair evaluations
// (Eq. 4, direct sum):
//   group g    : W i-blocks of 64 ions (one per warp, two ions per lane, packed FP32x2)
//   segment s  : j in [s n / S, (s+1) n / S), staged into shared memory
//   CTA g*S+s  : group g against segment s, and owner of the ions
//                [g0 + s |g| / S, g0 + (s+1) |g| / S) of its group
// A step: each warp leaves its (sum, compensation) pairs for (segment, ion) in global
// scratch; the S CTAs of a group count their arrivals on the group's counter; each
// owner merges its ions' S partials in segment order (Kahan), finishes the FP64 Verlet
// update (trap, drag and noise were evaluated before the pair loop), writes the next
// pair-stream entries and counts its CTA on the step counter; the next step starts once
// every CTA has counted.  The owners' FP64 state stays in registers from step to step.
// Every wait is bounded (2 s of %globaltimer) and gives up at once when another CTA has
// flagged a timeout, so a launch always ends.
//
// Summation order depends on (n, W, S) only: j ascending inside 128-wide chunks of a
// segment, chunks Kahan-added per warp, segments Kahan-merged in order.
#include <cstdio>

#include "iontrap_internal.cuh"

namespace it {

struct GpArgs {
  unsigned* sync;  // [0]: step arrivals of all CTAs; [32 (1 + g)]: arrivals of group g (zero between launches)
  long long K;     // steps in this launch
  int S;           // segments = CTAs per group
  int Lmax;        // entries per stream of the largest segment (shared-memory extent)
};

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait of a persistent form's poller until *ctr >= target: the counter alone is polled,
// the timeout flag and the clock every 64 polls.  ACQ: acquire loads (no fence needed
// after a successful wait).  Gives up (false) after limit ns, setting the timeout flag,
// or when another CTA has set it.
template <bool ACQ>
__device__ __noinline__ bool poll_wait(const unsigned* ctr, unsigned target, int* err, unsigned long long limit) {
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 1;; ++it) {
    unsigned c;
    if (ACQ)
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(ctr) : "memory");
    else
      c = ld_relaxed_u32(ctr);
    if (c >= target) return true;
    if ((it & 63) == 0) {
      if (*(volatile int*)err & ERR_TIMEOUT) return false;
      if (globaltimer_ns() - t0 > limit) {
        atomicOr(err, ERR_TIMEOUT);
        return false;
      }
    }
  }
}

// A CTA's arrival on a counter: release at GPU scope orders the CTA's earlier writes
// (after a CTA barrier) before the increment.
__device__ __forceinline__ void arrive_release(unsigned* ctr) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
}

// Trap spring constant of component c (the c-th value trap_springs gives, same roundings).
__device__ __forceinline__ double trap_spring_c(const TrapDev& tp, const SpeciesDev& sd, double cosv, int c) {
  if (tp.flags & IONTRAP_TRAP_OFF) return 0.0;
  if (tp.flags & IONTRAP_PSEUDO) return sd.ks[c];
  const double rwz2 = __dmul_rn(sd.rho, tp.wz2);
  const double rq4 = __dmul_rn(tp.q4, sd.rho);
  const double qc2 = __dmul_rn(2.0 * tp.q, cosv);
  const double ax = (c == 0) ? __dsub_rn(tp.a, qc2) : __dadd_rn(tp.a, qc2);
  const double kr = __fma_rn(rq4, ax, -0.5 * rwz2);
  return c == 2 ? rwz2 : kr;
}

template <int W>
__global__ void __launch_bounds__(32 * W, 16 / W) k_step_f32_gp(const __grid_constant__ StepArgs A, const GpArgs P) {
  constexpr int T = 32 * W;
  constexpr int B = 64;  // ions per warp
  // dynamic shared memory: segment hi[Lmax], lo[Lmax]; the owned ions' partials as
  // floats sum[3][S][R] and comp[3][S][R] (R <= Rmax = ceil(64 W / S)); the RF phase
  // cos(Omega t) at the force time of each of the K steps; the owned ions' drag
  // velocities [3][R] (laser cooling needs all three components of an ion)
  extern __shared__ __align__(16) float4 s_dyn[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long n = A.n;
  const int S = P.S;
  const unsigned G = gridDim.x;
  const int g = (int)blockIdx.x / S, s = (int)blockIdx.x % S;
  const long long g0 = (long long)g * (W * B), g1 = min(g0 + (long long)(W * B), n);
  const long long gs = g1 - g0;
  const long long r0 = g0 + (s * gs) / S, r1 = g0 + ((s + 1) * gs) / S;
  const int R = (int)(r1 - r0);
  const long long js0 = (s * n) / S, js1 = ((s + 1) * n) / S;
  const int L = (int)(js1 - js0);
  const long long i0 = g0 + (long long)warp * B;
  const int rmax = (64 * W + S - 1) / S;
  float4* sh = s_dyn;
  float4* sl = s_dyn + P.Lmax;
  float* fsum = reinterpret_cast<float*>(s_dyn + 2 * P.Lmax);
  float* fcmp = fsum + 3 * S * rmax;
  double* scos = reinterpret_cast<double*>(fcmp + 3 * S * rmax);  // 24 S rmax bytes past fsum: 8-byte aligned
  double* svd = scos + P.K;
  unsigned* ctr_step = P.sync;
  unsigned* ctr_grp = P.sync + 32 * (1 + g);
  const int poller = T - 1;
  const float4* part = reinterpret_cast<const float4*>(A.part);
  float4* wpart = reinterpret_cast<float4*>(A.part);
  const TrapDev& tp = A.trap;
  const long long ns0 = *A.step;
  const bool forces = A.mode == MODE_FORCES;  // one force evaluation of the current positions (K = 1)
  const unsigned long long lim = A.wait_ns ? A.wait_ns : kWaitLimitNs;
  const bool rf = !(tp.flags & (IONTRAP_RF_OFF | IONTRAP_TRAP_OFF | IONTRAP_PSEUDO));
  if (!forces)
    for (long long k = tid; k < P.K; k += T) scos[k] = rf ? cos(tp.Omega * ((double)(ns0 + k + 1) * tp.dt)) : 0.0;

  // owned items: thread k < 3R integrates component c = k / R of ion r0 + k % R, so the
  // FP64 chain of the integration is spread over three warps with a third of the
  // instructions each
  const int oc = tid / max(R, 1), oq = tid - oc * max(R, 1);
  const bool own = tid < 3 * R;
  const long long ie = r0 + oq;
  int spe = 0;
  double xf = 0.0, vd = 0.0;
  float z = 0.f;
  if (own) spe = A.sp[ie];
  if (own && !forces) {
    const double vh = half_kick(A.v[oc * n + ie], A.a[oc * n + ie], tp.hdt);
    vd = vh;
    xf = drift(A.x[oc * n + ie], vh, tp.dt);
  }
  // the Langevin normal of a step, drawn ahead of time (FP32 Box-Muller, as accel_ext)
  auto draw = [&](long long counter) {
    if (own && !forces && A.spc[spe].sigma > 0.0) {
      float zz[3];
      normals3_f32(tp.seed, counter, ie, zz);
      z = oc == 0 ? zz[0] : (oc == 1 ? zz[1] : zz[2]);
    }
  };
  draw(ns0 + 1);
  __syncthreads();

  for (long long t = 0; t < P.K; ++t) {
    const long long ns = ns0 + t;
    const int rb = forces ? (int)(ns & 1) : (int)((ns + 1) & 1);
    // positions x_{ns+1} are complete once every CTA has finished step t-1
    bool bad = false;
    if (t > 0 && tid == poller) {
      bad = !poll_wait<true>(ctr_step, G * (unsigned)t, A.err, lim);
    }
    if (__syncthreads_or(bad)) break;

    const float4* __restrict__ ghi = A.hi[rb];
    const float4* __restrict__ glo = A.lo[rb];
    for (int j = tid; j < L; j += T) {
      sh[j] = __ldcg(ghi + js0 + j);
      sl[j] = __ldcg(glo + js0 + j);
    }
    long long ii[2];
    float2 nxh[1][3], nxl[1][3];
    {
      float4 h[2], l[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        ii[k] = i0 + k * 32 + lane;
        h[k] = l[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ii[k] < n) {
          h[k] = __ldcg(ghi + ii[k]);
          l[k] = __ldcg(glo + ii[k]);
        }
      }
      nxh[0][0] = make_float2(-h[0].x, -h[1].x), nxh[0][1] = make_float2(-h[0].y, -h[1].y);
      nxh[0][2] = make_float2(-h[0].z, -h[1].z);
      nxl[0][0] = make_float2(-l[0].x, -l[1].x), nxl[0][1] = make_float2(-l[0].y, -l[1].y);
      nxl[0][2] = make_float2(-l[0].z, -l[1].z);
    }
    __syncthreads();  // segment staged

    if (i0 < n) {
      float ks[2][3], kc[2][3];
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) ks[k][d] = kc[k][d] = 0.0f;
      for (int c0 = 0; c0 < L; c0 += kSeg) {
        const int jn = min(kSeg, L - c0);
        const long long jc = js0 + c0;
        const bool diag = (jc < i0 + B) && (i0 < jc + jn);
        float2 acc[1][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[0][d] = make_float2(0.0f, 0.0f);
        if (A.unitw) {
          if (diag)
            segment_f32x2<2, true, true>(sh + c0, sl + c0, jn, jc, nxh, nxl, ii, acc);
          else
            segment_f32x2<2, false, true>(sh + c0, sl + c0, jn, jc, nxh, nxl, ii, acc);
        } else {
          if (diag)
            segment_f32x2<2, true>(sh + c0, sl + c0, jn, jc, nxh, nxl, ii, acc);
          else
            segment_f32x2<2, false>(sh + c0, sl + c0, jn, jc, nxh, nxl, ii, acc);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float a = k ? acc[0][d].y : acc[0][d].x;
            const float y = a - kc[k][d];
            const float tt = ks[k][d] + y;
            kc[k][d] = (tt - ks[k][d]) - y;
            ks[k][d] = tt;
          }
      }
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ii[k] < n) {
          const long long r = 2 * ((long long)s * n + ii[k]);
          __stcg(wpart + r, make_float4(ks[k][0], ks[k][1], ks[k][2], 0.0f));
          __stcg(wpart + r + 1, make_float4(kc[k][0], kc[k][1], kc[k][2], 0.0f));
        }
    }
    __syncthreads();
    if (tid == poller) {
      arrive_release(ctr_grp);
      bad = !poll_wait<true>(ctr_grp, (unsigned)S * (unsigned)(t + 1), A.err, lim);
    }
    // while the group's CTAs arrive: the owned components' force-independent terms
    // (trap, drag, laser, kick; the operations and order of accel_ext) and the next
    // step's normals
    double ext = 0.0;
    const float zk = z;
    if (own && !forces) {
      const SpeciesDev& sd = A.spc[spe];
      const double kc = trap_spring_c(tp, sd, scos[t], oc);
      ext = __fma_rn(-sd.gamma, vd, __dmul_rn(-kc, xf));
      if (tp.laser) svd[oc * R + oq] = vd;
    }
    if (t + 1 < P.K) draw(ns + 2);
    if (__syncthreads_or(bad)) break;
    if (own && !forces) {
      const SpeciesDev& sd = A.spc[spe];
      if (tp.laser && sd.lrate != 0.0) {
        const double v3[3] = {svd[oq], svd[R + oq], svd[2 * R + oq]};
        ext = __fma_rn(-laser_proj(sd, v3), sd.kdir[oc], ext);
      }
      if (sd.sigma > 0.0) ext = __fma_rn(sd.sigma, (double)zk, ext);
    }

    // the owned ions' S records, fetched by the whole CTA in one round trip
    for (int k = tid; k < R * S; k += T) {
      const int p = k / R, q = k - p * R;
      const long long r = 2 * ((long long)p * n + r0 + q);
      const float4 a = __ldcg(part + r), b = __ldcg(part + r + 1);
      fsum[(0 * S + p) * R + q] = a.x, fsum[(1 * S + p) * R + q] = a.y, fsum[(2 * S + p) * R + q] = a.z;
      fcmp[(0 * S + p) * R + q] = b.x, fcmp[(1 * S + p) * R + q] = b.y, fcmp[(2 * S + p) * R + q] = b.z;
    }
    __syncthreads();
    if (own) {  // merge in segment order (Kahan), then finish the step
      float su = 0.f, cu = 0.f;
      const float* ps = fsum + oc * S * R + oq;
      const float* pc = fcmp + oc * S * R + oq;
      constexpr int U = 8;
      for (int p0 = 0; p0 < S; p0 += U) {
        float a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (p0 + u < S) a[u] = ps[(p0 + u) * R], b[u] = pc[(p0 + u) * R];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (p0 + u < S) kahan_merge(su, cu, a[u], b[u]);
      }
      const double Sd = (double)cu - (double)su;
      const SpeciesDev& sd = A.spc[spe];
      if (forces) {
        A.out[oc * n + ie] = sd.coul * Sd;
      } else {
        const double acc = __fma_rn(sd.coul, Sd, ext);
        const double vn = half_kick(vd, acc, tp.hdt);
        const double vh = half_kick(vn, acc, tp.hdt);
        const double xn = drift(xf, vh, tp.dt);
        A.x[oc * n + ie] = xf;
        A.v[oc * n + ie] = vn;
        A.a[oc * n + ie] = acc;
        // next pair-stream entry, component by component (hi = fl(xn), lo = fl(xn - hi))
        const float h = __double2float_rn(xn);
        const float l = __double2float_rn(xn - (double)h);
        reinterpret_cast<float*>(A.hi[rb ^ 1] + ie)[oc] = h;
        reinterpret_cast<float*>(A.lo[rb ^ 1] + ie)[oc] = l;
        if (oc == 0) {
          reinterpret_cast<float*>(A.hi[rb ^ 1] + ie)[3] = sd.w;
          reinterpret_cast<float*>(A.lo[rb ^ 1] + ie)[3] = 0.0f;
        }
        if (!(isfinite(acc) && isfinite(vn) && isfinite(xn))) atomicOr(A.err, ERR_NONFINITE);
        vd = vh;  // the next step's kick and drift, as a fresh start would compute them
        xf = xn;
      }
    }
    __syncthreads();
    if (tid == poller && !(A.stall_on && (int)blockIdx.x == A.stall_cta && t == A.stall_step)) arrive_release(ctr_step);
  }

  // once every CTA has counted its last step: clear the counters, advance the step index
  // (not after a wait gave up: the handle's sticky timeout status retires it)
  if (blockIdx.x == 0 && tid == poller) {
    if (poll_wait<true>(ctr_step, G * (unsigned)P.K, A.err, lim)) {
      const int groups = (int)(G / (unsigned)S);
      for (int q = 0; q < groups; ++q) P.sync[32 * (1 + q)] = 0u;
      *ctr_step = 0u;
      if (!forces) *A.step = ns0 + P.K;
      __threadfence();
    }
  }
}

// Dynamic shared memory of a launch: the segment (2 Lmax float4), the owned ions'
// partials (2 x 3 x S x ceil(64 W / S) floats, rounded up to 16 bytes), K cosines and
// the owned ions' drag velocities (3 x ceil(64 W / S) doubles).
size_t gp_smem_bytes(int W, int S, int Lmax, long long K) {
  const size_t rmax = (size_t)((64 * W + S - 1) / S);
  const size_t recs = (6 * rmax * (size_t)S * sizeof(float) + 15) / 16 * 16;
  return 2 * (size_t)Lmax * sizeof(float4) + recs + (size_t)K * sizeof(double) + 3 * rmax * sizeof(double);
}

const void* gp_kernel(int W) {
  switch (W) {
    case 8: return (const void*)k_step_f32_gp<8>;
    case 16: return (const void*)k_step_f32_gp<16>;
    default: return nullptr;
  }
}

// Launch K steps of the grid-persistent form as one cooperative grid of G CTAs.
cudaError_t launch_gp(const StepArgs& a, unsigned* sync, int W, int S, int G, int Lmax, long long K,
                      cudaStream_t st) {
  const void* fn = gp_kernel(W);
  if (!fn) return cudaErrorInvalidValue;
  GpArgs P{sync, K, S, Lmax};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3((unsigned)(32 * W));
  cfg.dynamicSmemBytes = gp_smem_bytes(W, S, Lmax, K);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  StepArgs ac = a;
  void* params[] = {&ac, &P};
  return cudaLaunchKernelExC(&cfg, fn, params);
}

// Largest number of co-resident CTAs of the W-warp kernel with S segments of at most
// Lmax entries and up to max_k steps per launch.  The kernel's dynamic shared-memory
// limit is raised to the largest launch any handle may make (segments of max_lmax
// entries), so handles coexist.
int gp_max_ctas(int W, int S, int Lmax, int max_lmax, long long max_k, int sms) {
  const void* fn = gp_kernel(W);
  if (!fn || Lmax > max_lmax || S < 1) return 0;
  const size_t smem = gp_smem_bytes(W, S, Lmax, max_k);
  // ceil(64 W / S) S < 128 W; ceil(64 W / S) <= 64 W
  const size_t limit = 2 * (size_t)max_lmax * sizeof(float4) + 6 * 128 * (size_t)W * sizeof(float) + 16 +
                       (size_t)max_k * sizeof(double) + 3 * 64 * (size_t)W * sizeof(double);
  if (smem > limit) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) != cudaSuccess) return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 32 * W, smem) != cudaSuccess) return 0;
  return per * sms;
}

// ------------------------------------------------------------------ row-persistent form (fused = 5)
// One cooperative launch advances K steps.  CTA g owns the ions [g R, min((g+1) R, n)) and
// sums their Coulomb term over every j itself.  Its threads are laid out part-major:
// with one ion per thread (IPT = 1), thread t < R NP takes ion t % R against j-part t / R,
// the part p covering j in [p JP, (p+1) JP) (NP = 32 W / R parts, so nearly every thread
// works whatever R); with two (IPT = 2), thread t < RT NP (RT = ceil(R / 2)) takes the
// ions s and s + RT, s = t % RT, against part t / RT.  The j data of all parts is staged
// into shared memory as structure-of-arrays floats (four j per 16-byte shared load) and
// the pair loop runs two j at a time on packed FP32x2 instructions with an ion in both
// halves; a thread with two ions sums each of them that way against the same loaded j
// (half the shared-memory loads per pair; the loop stays bound by the FP32 pipe, and
// the choice between one and two ions per thread is the autotuner's).  The NP part
// partials (sum, compensation) of an ion merge in part order in shared memory, and one
// thread per owned ion component integrates it exactly as the grid-persistent form does.  One grid-wide step counter per
// step; no partial sum leaves the SM.  The next step's force-independent terms are
// evaluated right after the CTA has counted itself, while the others finish.
//
// Positions travel between steps in the same part-major layout the CTAs hold them in:
// besides the float4 pair stream, every owner writes its new position into a global copy
// of the staged arrays, so from the second step of a launch on one thread fetches them
// with bulk TMA copies of kRpBatches runs of consecutive parts, each completing on its own
// mbarrier, and a part's threads start as soon as their run has landed.  The CTA's own
// ions come from shared memory, where their owners left them.  The FP64 state and the
// float4 pair stream, which only the next launch reads, are written in a launch's last
// step (a launch stopped by a timeout leaves the state it started from).
//
// Summation order depends on (n, R, W, IPT) only: per part, j ascending in 128-j chunks
// summed as even and odd j (the two halves added), chunks Kahan-added; parts
// Kahan-merged in order.  Each (i, j) term is the same FP32 value as in
// the other forms.

struct RpArgs {
  unsigned* sync;  // [0]: step arrivals of all CTAs (zero between launches)
  long long K;     // steps in this launch
  int R;           // ions per CTA
  int NP;          // j-parts per CTA: 32 W / ceil(R / IPT)
  int JP;          // j entries per part: a multiple of 4 with JP / 4 odd (the parts of one
                   // warp read from distinct shared-memory banks); entries past n are padding
};

// Bulk copies (and mbarriers) per step: the parts are fetched in runs of about
// kRpRunBytes, at most kRpBatches of them (measured at N = 1024 .. 4096: 8 runs of 14 KB
// beat 4 of 29 KB, 4 runs of 15 KB beat 8 of 7.6 KB).
constexpr int kRpBatches = 8;
constexpr long long kRpRunBytes = 16 * 1024;

template <int W, int IPT>
__global__ void __launch_bounds__(32 * W, 1) k_step_f32_rp(const __grid_constant__ StepArgs A, const RpArgs P) {
  // dynamic shared memory: per part 7 x JP floats (SoA j data); partial sums and
  // compensations [NP][3][R] floats each; the RF phase of the K steps; the owned ions'
  // drag velocities [3][R] (laser cooling needs all three components of an ion); the
  // copy mbarriers; the owned ions' next positions [6][R] (hi x, y, z, lo x, y, z)
  extern __shared__ __align__(16) float4 s_dyn[];
  const int tid = threadIdx.x;
  const long long n = A.n;
  const unsigned G = gridDim.x;
  const int R = P.R, NP = P.NP, JP = P.JP;
  const long long r0 = (long long)blockIdx.x * R;
  const int Rg = (int)max(0LL, min((long long)R, n - r0));
  // one CTA holds every ion (n <= 3 * 32 W): the new positions go straight into its own
  // shared memory and the step ends at a CTA barrier -- no step counter, no poll, no bulk
  // copies
  const bool solo = G == 1u;
  float* sall = reinterpret_cast<float*>(s_dyn);
  float* ps = sall + (size_t)NP * 7 * JP;
  float* pc = ps + NP * 3 * R;
  // 28 NP JP + 24 NP R bytes in: a multiple of 8 (JP is a multiple of 4)
  double* scos = reinterpret_cast<double*>(pc + NP * 3 * R);
  double* svd = scos + P.K;
  uint64_t* bar = reinterpret_cast<uint64_t*>(svd + 3 * R);
  float* sself = reinterpret_cast<float*>(bar + kRpBatches);
  // global part-major copies of the staged arrays, one per pair-stream buffer
  const long long soa_len = (long long)NP * 7 * JP;
  float* gsoa = reinterpret_cast<float*>(A.part);
  const int nb = (int)min((long long)min(NP, kRpBatches),
                           max(1LL, (28LL * NP * JP + kRpRunBytes - 1) / kRpRunBytes));
  unsigned* ctr_step = P.sync;
  const int poller = 32 * W - 1;
  const TrapDev& tp = A.trap;
  const long long ns0 = *A.step;
  const bool forces = A.mode == MODE_FORCES;  // one force evaluation of the current positions (K = 1)
  const unsigned long long lim = A.wait_ns ? A.wait_ns : kWaitLimitNs;
  const bool rf = !(tp.flags & (IONTRAP_RF_OFF | IONTRAP_TRAP_OFF | IONTRAP_PSEUDO));
  for (long long k = tid; k < P.K; k += 32 * W) scos[k] = rf ? cos(tp.Omega * ((double)(ns0 + k + 1) * tp.dt)) : 0.0;
  if (tid == 0)
    for (int b = 0; b < nb; ++b) mbar_init(&bar[b], 1);
  // the padding entries of both global copies (their values never change); published to
  // the other CTAs by this CTA's first step arrival
  if (blockIdx.x == 0 && P.K > 1)
    for (long long e = n + tid; e < (long long)NP * JP; e += 32 * W) {
      const int p = (int)(e / JP), q = (int)(e - (long long)p * JP);
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        const float val = c < 3 ? 1e30f : 0.0f;
        gsoa[(long long)p * 7 * JP + c * JP + q] = val;
        gsoa[soa_len + (long long)p * 7 * JP + c * JP + q] = val;
      }
    }
  // every generic writer of data the copy engine reads fences against the async proxy
  if (blockIdx.x == 0 && P.K > 1) asm volatile("fence.proxy.async.global;" ::: "memory");

  // this thread's pair work: ion slot (slots slot and slot + RT with two ions per thread)
  // and j-part
  const int RT = (R + IPT - 1) / IPT;
  const int part = tid / RT, slot = tid - part * RT;
  const bool works = part < NP;
  const int ii = (int)(r0 + slot), ib = (int)(r0 + slot + RT);
  const bool hasb = IPT == 2 && slot + RT < Rg;
  const int mybatch = works ? ((part + 1) * nb - 1) / NP : 0;  // the copy run holding this part
  // owned items: thread k < 3 Rg integrates component c = k / Rg of ion r0 + k % Rg
  const int rq = max(Rg, 1);
  const int oc = tid / rq, oq = tid - oc * rq;
  const bool own = tid < 3 * Rg;
  const long long ie = r0 + oq;
  const long long iep = ie / JP;
  const long long ieo = iep * 7 * JP + (ie - iep * JP);  // ion ie's entry in a part-major copy
  int spe = 0;
  double xf = 0.0, vd = 0.0;
  float z = 0.f;
  if (own) spe = A.sp[ie];
  if (own && !forces) {
    const double vh = half_kick(A.v[oc * n + ie], A.a[oc * n + ie], tp.hdt);
    vd = vh;
    xf = drift(A.x[oc * n + ie], vh, tp.dt);
  }
  auto draw = [&](long long counter) {
    if (own && !forces && A.spc[spe].sigma > 0.0) {
      float zz[3];
      normals3_f32(tp.seed, counter, ie, zz);
      z = oc == 0 ? zz[0] : (oc == 1 ? zz[1] : zz[2]);
    }
  };
  // trap and drag of step t (the first operations of accel_ext); the velocity goes to
  // shared memory for the laser term
  auto ext_det = [&](long long t) -> double {
    const SpeciesDev& sd = A.spc[spe];
    const double kc = trap_spring_c(tp, sd, scos[t], oc);
    if (tp.laser) svd[oc * rq + oq] = vd;
    return __fma_rn(-sd.gamma, vd, __dmul_rn(-kc, xf));
  };
  // the charges of the owned ions into both global copies (they never change)
  if (own && !forces && oc == 0 && P.K > 1) {
    gsoa[ieo + 6 * JP] = A.spc[spe].w;
    gsoa[soa_len + ieo + 6 * JP] = A.spc[spe].w;
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncthreads();  // scos
  draw(ns0 + 1);
  double ext = own && !forces ? ext_det(0) : 0.0;
  float zk = z;
  if (P.K > 1) draw(ns0 + 2);
  __syncthreads();  // svd

  for (long long t = 0; t < P.K; ++t) {
    const long long ns = ns0 + t;
    const int rb = forces ? (int)(ns & 1) : (int)((ns + 1) & 1);
    bool bad = false;
    if (t > 0 && tid == poller && !solo) {
      bad = !poll_wait<true>(ctr_step, G * (unsigned)t, A.err, lim);
      if (!bad) {
        // the positions the other CTAs wrote (generic stores, ordered by the counter)
        // are read by the copy engine: a proxy fence orders them before the copies.  The
        // copies then overwrite shared memory that this CTA's threads last read before
        // the CTA barrier that preceded its arrival; the second fence orders those
        // generic accesses before the async writes as well.
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const float* src = gsoa + (rb ? soa_len : 0);
        for (int b = 0; b < nb; ++b) {
          const int p0 = b * NP / nb, p1 = (b + 1) * NP / nb;
          const uint32_t bytes = (uint32_t)((p1 - p0) * 7 * JP * sizeof(float));
          mbar_arrive_expect_tx(&bar[b], bytes);
          tma_bulk_g2s(sall + (size_t)p0 * 7 * JP, src + (size_t)p0 * 7 * JP, bytes, &bar[b]);
        }
      }
    }
    if (__syncthreads_or(bad)) break;
    // optional phase timestamps (iontrap_trace_step): 4 per CTA and step
    const long long tslot = ((long long)blockIdx.x * P.K + t) * 4;
    trace_mark(A.trace, tslot + 0);
    if (own && !forces) {  // the rest of accel_ext: laser, then the kick
      const SpeciesDev& sd = A.spc[spe];
      if (tp.laser && sd.lrate != 0.0) {
        const double v3[3] = {svd[oq], svd[rq + oq], svd[2 * rq + oq]};
        ext = __fma_rn(-laser_proj(sd, v3), sd.kdir[oc], ext);
      }
      if (sd.sigma > 0.0) ext = __fma_rn(sd.sigma, (double)zk, ext);
    }

    // positions x_{ns+1} of every part: entry e is j = e, part e / JP.  The first step of
    // a launch stages them from the pair stream; later steps wait for their copy run.
    float4 hi4 = make_float4(0.f, 0.f, 0.f, 0.f), lo4 = hi4, hib = hi4, lob = hi4;
    if (t == 0) {
      const float4* __restrict__ ghi = A.hi[rb];
      const float4* __restrict__ glo = A.lo[rb];
      for (int e = tid; e < NP * JP; e += 32 * W) {
        const int p = e / JP, q = e - p * JP;
        float4 h = make_float4(1e30f, 1e30f, 1e30f, 0.0f), l = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < n) {
          h = __ldcg(ghi + e);
          l = __ldcg(glo + e);
        }
        float* d = sall + (size_t)p * 7 * JP + q;
        d[0] = h.x, d[JP] = h.y, d[2 * JP] = h.z;
        d[3 * JP] = l.x, d[4 * JP] = l.y, d[5 * JP] = l.z;
        d[6 * JP] = h.w;
      }
      if (works && slot < Rg) {
        hi4 = __ldcg(ghi + ii);
        lo4 = __ldcg(glo + ii);
      }
      if (works && hasb) {
        hib = __ldcg(ghi + ib);
        lob = __ldcg(glo + ib);
      }
      __syncthreads();
    } else {
      if (works && slot < Rg) {
        hi4 = make_float4(sself[slot], sself[R + slot], sself[2 * R + slot], 0.f);
        lo4 = make_float4(sself[3 * R + slot], sself[4 * R + slot], sself[5 * R + slot], 0.f);
      }
      if (works && hasb) {
        const int sb = slot + RT;
        hib = make_float4(sself[sb], sself[R + sb], sself[2 * R + sb], 0.f);
        lob = make_float4(sself[3 * R + sb], sself[4 * R + sb], sself[5 * R + sb], 0.f);
      }
      if (works && !solo) bad = !mbar_wait_bounded(&bar[mybatch], (uint32_t)((t - 1) & 1), lim);
    }
    // each of the thread's ions in both halves of the packed registers
    float2 nh[IPT][3], nl[IPT][3];
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const float4 h = k ? hib : hi4, l = k ? lob : lo4;
      nh[k][0] = make_float2(-h.x, -h.x), nh[k][1] = make_float2(-h.y, -h.y), nh[k][2] = make_float2(-h.z, -h.z);
      nl[k][0] = make_float2(-l.x, -l.x), nl[k][1] = make_float2(-l.y, -l.y), nl[k][2] = make_float2(-l.z, -l.z);
    }
    trace_mark(A.trace, tslot + 1);

    if (works && !bad) {
      const float* sj = sall + (size_t)part * 7 * JP;
      // Kahan sums of the chunks, per ion of the thread ([0]: ion a, [1]: ion b)
      float ks[IPT][3], kcp[IPT][3];
#pragma unroll
      for (int k = 0; k < IPT; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) ks[k][d] = kcp[k][d] = 0.f;
      for (int c0 = 0; c0 < JP; c0 += kSeg) {
        const int qn = min(kSeg, JP - c0);
        float2 acc[IPT][3];  // per ion: even and odd j
#pragma unroll
        for (int k = 0; k < IPT; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) acc[k][d] = make_float2(0.f, 0.f);
        // the self pair can only sit in a chunk that overlaps the CTA's own ions; the
        // variant is chosen per warp (its lanes may belong to two parts)
        const int jc = part * JP + c0;
        const bool diag = __any_sync(__activemask(), (jc < r0 + Rg) && (r0 < jc + qn));
        if constexpr (IPT == 1) {
          if (A.unitw) {
            if (diag)
              rp_chunk<true, true>(sj + c0, sj + 6 * JP + c0, JP, qn, jc, ii, nh[0], nl[0], acc[0]);
            else
              rp_chunk<false, true>(sj + c0, sj + 6 * JP + c0, JP, qn, jc, ii, nh[0], nl[0], acc[0]);
          } else {
            if (diag)
              rp_chunk<true, false>(sj + c0, sj + 6 * JP + c0, JP, qn, jc, ii, nh[0], nl[0], acc[0]);
            else
              rp_chunk<false, false>(sj + c0, sj + 6 * JP + c0, JP, qn, jc, ii, nh[0], nl[0], acc[0]);
          }
        } else {
          if (A.unitw) {
            if (diag)
              rp_chunk_i2<true, true>(sj + c0, sj + 6 * JP + c0, JP, qn, jc, ii, ib, nh, nl, acc);
            else
              rp_chunk_i2<false, true>(sj + c0, sj + 6 * JP + c0, JP, qn, jc, ii, ib, nh, nl, acc);
          } else {
            if (diag)
              rp_chunk_i2<true, false>(sj + c0, sj + 6 * JP + c0, JP, qn, jc, ii, ib, nh, nl, acc);
            else
              rp_chunk_i2<false, false>(sj + c0, sj + 6 * JP + c0, JP, qn, jc, ii, ib, nh, nl, acc);
          }
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            // the even and odd j of the chunk added
            const float a = acc[k][d].x + acc[k][d].y;
            const float y = a - kcp[k][d];
            const float tt = ks[k][d] + y;
            kcp[k][d] = (tt - ks[k][d]) - y;
            ks[k][d] = tt;
          }
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        ps[(part * 3 + d) * R + slot] = ks[0][d];
        pc[(part * 3 + d) * R + slot] = kcp[0][d];
        if (IPT == 2 && slot + RT < R) {
          ps[(part * 3 + d) * R + slot + RT] = ks[IPT - 1][d];
          pc[(part * 3 + d) * R + slot + RT] = kcp[IPT - 1][d];
        }
      }
    }
    if (__syncthreads_or(bad)) {  // a copy run never landed: flag, let every copy finish, stop
      if (tid == poller) {
        atomicOr(A.err, ERR_TIMEOUT);
        for (int b = 0; b < nb; ++b) mbar_wait_bounded(&bar[b], (uint32_t)((t - 1) & 1), lim);
      }
      __syncthreads();
      break;
    }
    trace_mark(A.trace, tslot + 2);

    if (own) {  // merge in part order (Kahan), then finish the step
      float su = 0.f, cu = 0.f;
      for (int p = 0; p < NP; ++p) kahan_merge(su, cu, ps[(p * 3 + oc) * R + oq], pc[(p * 3 + oc) * R + oq]);
      const double Sd = (double)cu - (double)su;
      const SpeciesDev& sd = A.spc[spe];
      if (forces) {
        A.out[oc * n + ie] = sd.coul * Sd;
      } else {
        const double acc = __fma_rn(sd.coul, Sd, ext);
        const double vn = half_kick(vd, acc, tp.hdt);
        const double vh = half_kick(vn, acc, tp.hdt);
        const double xn = drift(xf, vh, tp.dt);
        const float h = __double2float_rn(xn);
        const float l = __double2float_rn(xn - (double)h);
        if (t + 1 == P.K) {  // the launch's last step: FP64 state and the pair stream
          A.x[oc * n + ie] = xf;
          A.v[oc * n + ie] = vn;
          A.a[oc * n + ie] = acc;
          reinterpret_cast<float*>(A.hi[rb ^ 1] + ie)[oc] = h;
          reinterpret_cast<float*>(A.lo[rb ^ 1] + ie)[oc] = l;
          if (oc == 0) {
            reinterpret_cast<float*>(A.hi[rb ^ 1] + ie)[3] = sd.w;
            reinterpret_cast<float*>(A.lo[rb ^ 1] + ie)[3] = 0.0f;
          }
        } else if (solo) {  // the next step's positions, in place (every read of them is done)
          sall[ieo + oc * JP] = h;
          sall[ieo + (3 + oc) * JP] = l;
          sself[oc * R + oq] = h;
          sself[(3 + oc) * R + oq] = l;
        } else {  // the next step's copies: part-major global, own ions in shared
          float* g = gsoa + (rb ? 0 : soa_len) + ieo;
          g[oc * JP] = h;
          g[(3 + oc) * JP] = l;
          sself[oc * R + oq] = h;
          sself[(3 + oc) * R + oq] = l;
          asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        // a non-finite acceleration or velocity reaches xn = xf + dt (vn + dt/2 acc)
        if (!isfinite(xn)) atomicOr(A.err, ERR_NONFINITE);
        vd = vh;
        xf = xn;
      }
    }
    __syncthreads();
    trace_mark(A.trace, tslot + 3);
    if (tid == poller && !solo && !(A.stall_on && (int)blockIdx.x == A.stall_cta && t == A.stall_step))
      arrive_release(ctr_step);
    // the next step's trap and drag and the noise after it, while the other CTAs finish
    if (t + 1 < P.K && !forces) {
      if (own) ext = ext_det(t + 1);
      zk = z;
      if (t + 2 < P.K) draw(ns + 3);
    }
  }

  // once every CTA has counted its last step: clear the counter, advance the step index.
  // A launch that gave up on a wait leaves both alone: its FP64 state is still the one it
  // started from, and the handle's sticky timeout status retires the counter with it.
  if (blockIdx.x == 0 && tid == poller) {
    if (solo || poll_wait<true>(ctr_step, G * (unsigned)P.K, A.err, lim)) {
      *ctr_step = 0u;
      if (!forces) *A.step = ns0 + P.K;
      __threadfence();
    }
  }
}

// Dynamic shared memory of a launch: the parts' SoA j data (NP x 7 x JP floats), the part
// partials (2 x NP x 3 x R floats), K cosines, 3 R drag velocities, the copy mbarriers and
// the owned ions' next positions (6 R floats).
size_t rp_smem_bytes(int W, int R, int NP, int JP, long long K) {
  (void)W;
  const size_t parts = (size_t)NP * 7 * JP * sizeof(float);
  const size_t recs = 2 * (size_t)NP * 3 * R * sizeof(float);
  return parts + recs + (size_t)K * sizeof(double) + 3 * (size_t)R * sizeof(double) +
         kRpBatches * sizeof(uint64_t) + 6 * (size_t)R * sizeof(float);
}

// Global scratch of a launch: the two part-major position copies (NP x 7 x JP floats each).
size_t rp_scratch_bytes(int NP, int JP) { return 2 * (size_t)NP * 7 * JP * sizeof(float); }

const void* rp_kernel(int W, int I) {
  if (I == 1) return W == 8 ? (const void*)k_step_f32_rp<8, 1> : W == 16 ? (const void*)k_step_f32_rp<16, 1> : nullptr;
  if (I == 2) return W == 8 ? (const void*)k_step_f32_rp<8, 2> : W == 16 ? (const void*)k_step_f32_rp<16, 2> : nullptr;
  return nullptr;
}

// Co-resident CTAs of a launch shape (W warps, I ions per thread) with up to max_k steps
// per launch (the kernel's dynamic shared-memory limit is raised to 227 KB once, so
// handles coexist).
int rp_max_ctas(int W, int R, int NP, int JP, int I, long long max_k, int sms) {
  const void* fn = rp_kernel(W, I);
  if (!fn) return 0;
  const size_t smem = rp_smem_bytes(W, R, NP, JP, max_k);
  if (smem > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess) return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 32 * W, smem) != cudaSuccess) return 0;
  return per * sms;
}

cudaError_t launch_rp(const StepArgs& a, unsigned* sync, int W, int R, int NP, int JP, int I, int G, long long K,
                      cudaStream_t st) {
  const void* fn = rp_kernel(W, I);
  if (!fn) return cudaErrorInvalidValue;
  RpArgs P{sync, K, R, NP, JP};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3((unsigned)(32 * W));
  cfg.dynamicSmemBytes = rp_smem_bytes(W, R, NP, JP, K);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  StepArgs ac = a;
  void* params[] = {&ac, &P};
  return cudaLaunchKernelExC(&cfg, fn, params);
}

}  // namespace it
