// iontrap_internal.cuh -- device-side building blocks of libiontrap.so (sm_103a).
//
// Shared by the kernels of this library only.  The FP64 oracle under oracle/ is a
// separate program and shares nothing with this file.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "iontrap.h"

namespace it {

// CODATA 2018 (e, k_B exact).
constexpr double kE = 1.602176634e-19;
constexpr double kKB = 1.380649e-23;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kPi = 3.14159265358979323846;

// Segment of the j-range summed plainly in FP32 before its sum is added into the
// compensated per-ion accumulator.
constexpr int kSeg = 128;

enum Mode : int { MODE_STEP = 0, MODE_INIT = 1, MODE_FORCES = 2 };
enum ErrBits : int { ERR_NONFINITE = 1, ERR_TIMEOUT = 2 };

// Per-species constants, precomputed on the host in FP64.
struct SpeciesDev {
  double coul;   // k_e e^2 z / M: Coulomb acceleration per unit of sum_j z_j d/r^3
  double rho;    // (z/M) / (z_0/M_0): scales a, q and omega_z^2 of species 0
  double gamma;  // Langevin rate of this species' bath (1/dampingTime), 1/s
  double sigma;  // sqrt(2 gamma k_B T / (M dt)): std. dev. of the Langevin kick acceleration
  double lrate;  // laser-cooling rate |g|, 1/s (0: no laser on this species)
  double kdir[3];  // laser direction g / |g|
  double ks[3];  // static spring constants of the pseudopotential trap (IONTRAP_PSEUDO), 1/s^2
  double mass;   // kg
  double z;      // charge number
  float w;       // z as float, the source weight in the FP32 pair stream
  float pad;
};

struct TrapDev {
  double dt, hdt;      // step and half step
  double Omega, q4;    // RF angular frequency and Omega^2/4
  double a, q, wz2;    // Mathieu a, q and omega_z^2 of species 0
  unsigned long long seed;
  unsigned flags;
  int laser;           // some species is laser-cooled
};

// Arguments of one force+integrate launch.  All per-ion arrays are SoA [3][n].
struct StepArgs {
  long long n;
  float4* hi[2];       // FP32 form: (x_hi, y_hi, z_hi, z_charge), ping-pong
  float4* lo[2];       // FP32 form: (x_lo, y_lo, z_lo, 0),  x = x_hi + x_lo
  double4_32a* p64[2];     // FP64 form: (x, y, z, z_charge), ping-pong
  double* x;           // positions x_n
  double* v;           // velocities v_n
  double* a;           // accelerations a_n
  const unsigned char* sp;  // species index per ion
  void* part;          // per-split partial sums (scratch)
  unsigned* cnt;       // per-i-block arrival counters (scratch, zero between launches)
  unsigned* done;      // completed i-blocks (scratch, zero between launches)
  long long* step;     // state step index n (device resident)
  int* err;            // ErrBits, sticky
  double* out;         // MODE_FORCES output [3][n]
  unsigned long long* trace;  // optional per-CTA phase timestamps (globaltimer ns), or null
  long long trace_epi;        // offset of the epilogue kernel's marks in trace
  int mode;
  int unitw;           // every ion has charge +1 e: the pair loop skips the z_j factor (exact)
  int jsplit;          // j-range per CTA (grid.y = ceil(n / jsplit))
  int nsplit;          // ceil(n / jsplit): partials per ion for the epilogue kernel
  // failure-detection test hook of the persistent forms (iontrap_test_stall): when
  // stall_on, CTA stall_cta withholds its arrival on the grid-wide step counter at step
  // stall_step of every launch, so that the other CTAs' bounded waits expire
  int stall_on;
  int stall_cta;
  long long stall_step;
  unsigned long long wait_ns;  // limit of the persistent forms' bounded waits (0: kWaitLimitNs)
  TrapDev trap;
  SpeciesDev spc[IONTRAP_MAX_SPECIES];
};

// One ensemble of a batched launch (FP32 form, resident in shared memory).
struct BatchEns {
  double* x;            // handle state, SoA [3][n]
  double* v;
  double* a;
  const unsigned char* sp;
  float4* hi[2];        // the handle's pair streams (read at start, refreshed at the end)
  float4* lo[2];
  long long* step;      // the handle's device step counter
  int* err;
  long long n;
  long long step0;      // state step index when the batch was enqueued
  long long remaining;  // steps still to take; decremented by the kernel
  int nspecies;
  int unitw;            // every ion has charge +1 e
  TrapDev trap;
  SpeciesDev spc[IONTRAP_MAX_SPECIES];
};

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk (non-tensor) TMA copy global -> shared, completing on an mbarrier.  Both
// addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for an mbarrier phase, giving up after limit_ns of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

// Phase timestamp of this CTA into the optional trace buffer (thread 0 only).
__device__ __forceinline__ void trace_mark(unsigned long long* trace, long long slot) {
  if (trace && threadIdx.x == 0) trace[slot] = globaltimer_ns();
}

// ------------------------------------------------------------------ FP32 pair terms
// d = x_j - x_i from hi/lo pairs, with the i side held negated in registers:
// (x_j,hi - x_i,hi) is exact for close pairs (Sterbenz) and the lo difference restores
// the bits FP32 rounding dropped from both positions.  The accumulators therefore hold
// -sum_j z_j (x_i - x_j)/r^3; the epilogue flips the sign.
template <int I, bool DIAG, bool UNITW = false>
__device__ __forceinline__ void segment_f32(const float4* __restrict__ sh, const float4* __restrict__ sl, int jn,
                                            long long jbase, const float (&nxh)[I][3], const float (&nxl)[I][3],
                                            const long long (&ii)[I], float (&acc)[I][3]) {
#pragma unroll 4
  for (int j = 0; j < jn; ++j) {
    const float4 ph = sh[j];
    const float4 pl = sl[j];
#pragma unroll
    for (int k = 0; k < I; ++k) {
      const float dx = (ph.x + nxh[k][0]) + (pl.x + nxl[k][0]);
      const float dy = (ph.y + nxh[k][1]) + (pl.y + nxl[k][1]);
      const float dz = (ph.z + nxh[k][2]) + (pl.z + nxl[k][2]);
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      float ri = rsqrt_approx(r2);
      if (DIAG) ri = (jbase + j == ii[k]) ? 0.0f : ri;
      const float ri2 = ri * ri;
      const float s = (UNITW ? ri : ph.w * ri) * ri2;  // z_j / r^3 (z_j = 1: the product is exact)
      acc[k][0] = fmaf(s, dx, acc[k][0]);
      acc[k][1] = fmaf(s, dy, acc[k][1]);
      acc[k][2] = fmaf(s, dz, acc[k][2]);
    }
  }
}

// The same arithmetic on two ions per instruction (packed FP32x2 FADD/FMUL/FFMA of
// sm_100+); each lane rounds exactly as the scalar loop does, so both loops give the
// same bits.
template <int I, bool DIAG, bool UNITW = false>
__device__ __forceinline__ void segment_f32x2(const float4* __restrict__ sh, const float4* __restrict__ sl, int jn,
                                              long long jbase, const float2 (&nxh)[I / 2][3],
                                              const float2 (&nxl)[I / 2][3], const long long (&ii)[I],
                                              float2 (&acc)[I / 2][3]) {
#pragma unroll 4
  for (int j = 0; j < jn; ++j) {
    const float4 ph = sh[j];
    const float4 pl = sl[j];
    const float2 hx = make_float2(ph.x, ph.x), hy = make_float2(ph.y, ph.y), hz = make_float2(ph.z, ph.z);
    const float2 lx = make_float2(pl.x, pl.x), ly = make_float2(pl.y, pl.y), lz = make_float2(pl.z, pl.z);
    const float2 w = make_float2(ph.w, ph.w);
#pragma unroll
    for (int k = 0; k < I / 2; ++k) {
      const float2 dx = __fadd2_rn(__fadd2_rn(hx, nxh[k][0]), __fadd2_rn(lx, nxl[k][0]));
      const float2 dy = __fadd2_rn(__fadd2_rn(hy, nxh[k][1]), __fadd2_rn(ly, nxl[k][1]));
      const float2 dz = __fadd2_rn(__fadd2_rn(hz, nxh[k][2]), __fadd2_rn(lz, nxl[k][2]));
      const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
      float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
      if (DIAG) {
        ri.x = (jbase + j == ii[2 * k]) ? 0.0f : ri.x;
        ri.y = (jbase + j == ii[2 * k + 1]) ? 0.0f : ri.y;
      }
      const float2 ri2 = __fmul2_rn(ri, ri);
      const float2 s = __fmul2_rn(UNITW ? ri : __fmul2_rn(w, ri), ri2);
      acc[k][0] = __ffma2_rn(s, dx, acc[k][0]);
      acc[k][1] = __ffma2_rn(s, dy, acc[k][1]);
      acc[k][2] = __ffma2_rn(s, dz, acc[k][2]);
    }
  }
}

// ------------------------------------------------------------------ part-major pair loop
// The row-persistent form and the clustered batched form hold the j data of a CTA as
// structure-of-arrays floats in shared memory, in parts of JP entries (rows x_hi, y_hi,
// z_hi, x_lo, y_lo, z_lo, z at stride JP).  A thread sums one ion against one part, two j
// per packed instruction with its ion in both halves of its registers.
// Pair terms of one thread's ion against two j (packed); DIAG: the self pair is excluded
// by its index (only chunks that may hold it take this variant).
template <bool DIAG, bool UNITW>
__device__ __forceinline__ void rp_pair2(float2 hx, float2 hy, float2 hz, float2 lx, float2 ly, float2 lz, float2 w,
                                         int j, int i, const float2 (&nh)[3], const float2 (&nl)[3],
                                         float2 (&acc)[3]) {
  const float2 dx = __fadd2_rn(__fadd2_rn(hx, nh[0]), __fadd2_rn(lx, nl[0]));
  const float2 dy = __fadd2_rn(__fadd2_rn(hy, nh[1]), __fadd2_rn(ly, nl[1]));
  const float2 dz = __fadd2_rn(__fadd2_rn(hz, nh[2]), __fadd2_rn(lz, nl[2]));
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
  if (DIAG) {
    ri.x = (j == i) ? 0.0f : ri.x;
    ri.y = (j + 1 == i) ? 0.0f : ri.y;
  }
  const float2 ri2 = __fmul2_rn(ri, ri);
  const float2 s = UNITW ? __fmul2_rn(ri, ri2) : __fmul2_rn(__fmul2_rn(w, ri), ri2);
  acc[0] = __ffma2_rn(s, dx, acc[0]);
  acc[1] = __ffma2_rn(s, dy, acc[1]);
  acc[2] = __ffma2_rn(s, dz, acc[2]);
}

// qn (a multiple of 4) staged j of one part (stride JP between x_hi, y_hi, z_hi, x_lo,
// y_lo, z_lo; the charges z from sw), four j per iteration from 16-byte shared loads.
// Padding entries sit at 1e30 m: r^2 overflows to infinity, rsqrt gives 0, the term is
// exactly 0.
template <bool DIAG, bool UNITW>
__device__ __forceinline__ void rp_chunk(const float* __restrict__ sj, const float* __restrict__ sw, int JP, int qn,
                                         int jbase, int i, const float2 (&nh)[3], const float2 (&nl)[3],
                                         float2 (&acc)[3]) {
#pragma unroll 2
  for (int q = 0; q < qn; q += 4) {
    const float4 hx = *reinterpret_cast<const float4*>(sj + q);
    const float4 hy = *reinterpret_cast<const float4*>(sj + JP + q);
    const float4 hz = *reinterpret_cast<const float4*>(sj + 2 * JP + q);
    const float4 lx = *reinterpret_cast<const float4*>(sj + 3 * JP + q);
    const float4 ly = *reinterpret_cast<const float4*>(sj + 4 * JP + q);
    const float4 lz = *reinterpret_cast<const float4*>(sj + 5 * JP + q);
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!UNITW) w = *reinterpret_cast<const float4*>(sw + q);
    rp_pair2<DIAG, UNITW>(make_float2(hx.x, hx.y), make_float2(hy.x, hy.y), make_float2(hz.x, hz.y),
                    make_float2(lx.x, lx.y), make_float2(ly.x, ly.y), make_float2(lz.x, lz.y), make_float2(w.x, w.y),
                    jbase + q, i, nh, nl, acc);
    rp_pair2<DIAG, UNITW>(make_float2(hx.z, hx.w), make_float2(hy.z, hy.w), make_float2(hz.z, hz.w),
                    make_float2(lx.z, lx.w), make_float2(ly.z, ly.w), make_float2(lz.z, lz.w), make_float2(w.z, w.w),
                    jbase + q + 2, i, nh, nl, acc);
  }
}

// Two ions per thread: the j data loaded from shared memory serves both ions, each summed
// exactly as rp_chunk sums one (two j per packed instruction with the ion in both halves;
// acc[k] holds ion k's even and odd j).
template <bool DIAG, bool UNITW>
__device__ __forceinline__ void rp_chunk_i2(const float* __restrict__ sj, const float* __restrict__ sw, int JP, int qn,
                                            int jbase, int ia, int ib, const float2 (&nh)[2][3],
                                            const float2 (&nl)[2][3], float2 (&acc)[2][3]) {
#pragma unroll 1
  for (int q = 0; q < qn; q += 4) {
    const float4 hx = *reinterpret_cast<const float4*>(sj + q);
    const float4 hy = *reinterpret_cast<const float4*>(sj + JP + q);
    const float4 hz = *reinterpret_cast<const float4*>(sj + 2 * JP + q);
    const float4 lx = *reinterpret_cast<const float4*>(sj + 3 * JP + q);
    const float4 ly = *reinterpret_cast<const float4*>(sj + 4 * JP + q);
    const float4 lz = *reinterpret_cast<const float4*>(sj + 5 * JP + q);
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!UNITW) w = *reinterpret_cast<const float4*>(sw + q);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int i = k ? ib : ia;
      rp_pair2<DIAG, UNITW>(make_float2(hx.x, hx.y), make_float2(hy.x, hy.y), make_float2(hz.x, hz.y),
                            make_float2(lx.x, lx.y), make_float2(ly.x, ly.y), make_float2(lz.x, lz.y),
                            make_float2(w.x, w.y), jbase + q, i, nh[k], nl[k], acc[k]);
      rp_pair2<DIAG, UNITW>(make_float2(hx.z, hx.w), make_float2(hy.z, hy.w), make_float2(hz.z, hz.w),
                            make_float2(lx.z, lx.w), make_float2(ly.z, ly.w), make_float2(lz.z, lz.w),
                            make_float2(w.z, w.w), jbase + q + 2, i, nh[k], nl[k], acc[k]);
    }
  }
}

// ------------------------------------------------------------------ split partials
// RF phase at the force time of a launch in the given mode.
__device__ __forceinline__ double force_time_cos(const StepArgs& A, long long ns) {
  const long long nf = (A.mode == MODE_STEP) ? ns + 1 : ns;
  if (A.trap.flags & (IONTRAP_RF_OFF | IONTRAP_TRAP_OFF | IONTRAP_PSEUDO)) return 0.0;
  return cos(A.trap.Omega * ((double)nf * A.trap.dt));
}

// Split partials are stored as one 32-byte record per (split, ion):
//   FP32 form: float[8] = (sum_x, sum_y, sum_z, 0, comp_x, comp_y, comp_z, 0)
//   FP64 form: double[4] = (sum_x, sum_y, sum_z, 0)
// at record index split * n + i.  The merge runs in split order: FP32 form by
// compensated (Kahan) addition of the (sum, compensation) pairs -- the accumulators hold
// the negated sum, hence the sign -- FP64 form by a plain FP64 sum.
__device__ __forceinline__ void kahan_merge(float& s, float& cc, float ps, float pc) {
  const float y = ps - cc;
  const float t = s + y;
  cc = ((t - s) - y) + pc;
  s = t;
}

__device__ __forceinline__ void merge_f32(const float4* __restrict__ part, long long n, long long i, int nsplit,
                                          double S[3]) {
  float s[3] = {0.f, 0.f, 0.f}, cc[3] = {0.f, 0.f, 0.f};
  constexpr int U = 4;
  for (int p0 = 0; p0 < nsplit; p0 += U) {
    float4 a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (p0 + u < nsplit) {
        a[u] = __ldcg(part + 2 * ((p0 + u) * n + i));
        b[u] = __ldcg(part + 2 * ((p0 + u) * n + i) + 1);
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (p0 + u < nsplit) {
        kahan_merge(s[0], cc[0], a[u].x, b[u].x);
        kahan_merge(s[1], cc[1], a[u].y, b[u].y);
        kahan_merge(s[2], cc[2], a[u].z, b[u].z);
      }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) S[c] = (double)cc[c] - (double)s[c];
}

// ------------------------------------------------------------------ Philox-4x64-10
// Salmon et al., SC'11: ten rounds of two 64x64 -> 128-bit products; key bumped by the
// Weyl constants between rounds.
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

// Three standard normals for (seed, counter, id): u_k = (top 23 bits + 1/2) 2^-23 (exact
// in FP32), Box-Muller on (u0, u1) and (u2, u3).  FP32 arithmetic (the FP32 form's noise).
__device__ __forceinline__ void normals3_f32(unsigned long long seed, long long counter, long long id,
                                             float z[3]) {
  unsigned long long c[4] = {(unsigned long long)counter, (unsigned long long)id, 0ull, 0ull};
  philox4x64_10(c, seed, 0ull);
  float u[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) u[k] = ((float)(unsigned)(c[k] >> 41) + 0.5f) * 0x1p-23f;
  const float r1 = sqrtf(-2.0f * logf(u[0]));
  const float r2 = sqrtf(-2.0f * logf(u[2]));
  float s1, c1, s2, c2;
  sincospif(2.0f * u[1], &s1, &c1);
  sincospif(2.0f * u[3], &s2, &c2);
  z[0] = r1 * c1;
  z[1] = r1 * s1;
  z[2] = r2 * c2;
}

// The same three normals in FP64 arithmetic (the plain FP64 form's noise).
__device__ __forceinline__ void normals3_f64(unsigned long long seed, long long counter, long long id,
                                             double z[3]) {
  unsigned long long c[4] = {(unsigned long long)counter, (unsigned long long)id, 0ull, 0ull};
  philox4x64_10(c, seed, 0ull);
  double u[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) u[k] = ((double)(c[k] >> 41) + 0.5) * 0x1p-23;
  const double r1 = sqrt(-2.0 * log(u[0]));
  const double r2 = sqrt(-2.0 * log(u[2]));
  double s1, c1, s2, c2;
  sincospi(2.0 * u[1], &s1, &c1);
  sincospi(2.0 * u[3], &s2, &c2);
  z[0] = r1 * c1;
  z[1] = r1 * s1;
  z[2] = r2 * c2;
}

// ------------------------------------------------------------------ integrator pieces
// Written with explicit FMAs so that the drift the epilogue applies when it writes the
// next pair stream and the one it re-applies at the start of the next step are the same
// operations, hence the same bits.
__device__ __forceinline__ double half_kick(double v, double a, double hdt) { return __fma_rn(hdt, a, v); }
__device__ __forceinline__ double drift(double x, double vh, double dt) { return __fma_rn(dt, vh, x); }

// Entry i of pair stream b for the next positions xn (FP64 form: double4_32a; FP32 form:
// hi = fl(xn), lo = fl(xn - hi)).
template <bool F64>
__device__ __forceinline__ void write_pair(const StepArgs& A, int b, long long i, const double xn[3], float w) {
  if (F64) {
    A.p64[b][i] = make_double4_32a(xn[0], xn[1], xn[2], (double)w);
  } else {
    float h[3], l[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h[c] = __double2float_rn(xn[c]);
      l[c] = __double2float_rn(xn[c] - (double)h[c]);
    }
    A.hi[b][i] = make_float4(h[0], h[1], h[2], w);
    A.lo[b][i] = make_float4(l[0], l[1], l[2], 0.0f);
  }
}

// Trap spring constants of one species at force time (RF phase cosv): the trap
// acceleration is (-kx x, -ky y, -kz z).  Computed once per species per step.
__device__ __forceinline__ void trap_springs(const TrapDev& tp, const SpeciesDev& sd, double cosv, double k[3]) {
  if (tp.flags & IONTRAP_TRAP_OFF) {
    k[0] = k[1] = k[2] = 0.0;
    return;
  }
  if (tp.flags & IONTRAP_PSEUDO) {  // static pseudopotential springs (Eq. 2 or given frequencies)
    k[0] = sd.ks[0], k[1] = sd.ks[1], k[2] = sd.ks[2];
    return;
  }
  const double rwz2 = __dmul_rn(sd.rho, tp.wz2);
  const double rq4 = __dmul_rn(tp.q4, sd.rho);
  const double qc2 = __dmul_rn(2.0 * tp.q, cosv);
  k[0] = __fma_rn(rq4, __dsub_rn(tp.a, qc2), -0.5 * rwz2);
  k[1] = __fma_rn(rq4, __dadd_rn(tp.a, qc2), -0.5 * rwz2);
  k[2] = rwz2;
}

// Acceleration of one ion at force time, FP64 in both forms, split in two so that the
// part that does not depend on the Coulomb sum can be evaluated before the sum is known:
//   ext = -k xf - gamma vd - lrate (kdir.vd) kdir + sigma xi(seed, counter, id)  (accel_ext)
//   acc = k_e e^2 z/M S + ext                                                  (accel_total)
// with k the spring constants, gamma and sigma the bath and (lrate, kdir) the laser of the
// ion's species, and S = sum_j z_j d/r^3.  Explicit
// roundings (no FMA contraction left to the compiler): every kernel produces the same
// bits.  The trajectories of these clouds amplify FP32-sized perturbations of the RF trap
// term by ~1e4 within 100 steps, so no term is evaluated in FP32.  F64 selects FP64
// Box-Muller noise.
// The deterministic part (trap springs and drag) and the kick sigma*xi, separately so
// that a kernel can draw the normals ahead of time.
// Laser-cooling drag of one ion (laserCool, Sec. 3 "Cooling the motion of ions"): the
// rate times the drag velocity's projection on the beam direction, -lrate (k.vd) k.
__device__ __forceinline__ double laser_proj(const SpeciesDev& sd, const double vd[3]) {
  const double kv = __fma_rn(sd.kdir[2], vd[2], __fma_rn(sd.kdir[1], vd[1], __dmul_rn(sd.kdir[0], vd[0])));
  return __dmul_rn(sd.lrate, kv);
}

__device__ __forceinline__ void accel_ext_det(const SpeciesDev& sd, const double k[3], const double xf[3],
                                              const double vd[3], double ext[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) ext[c] = __fma_rn(-sd.gamma, vd[c], __dmul_rn(-k[c], xf[c]));
  if (sd.lrate != 0.0) {
    const double lp = laser_proj(sd, vd);
#pragma unroll
    for (int c = 0; c < 3; ++c) ext[c] = __fma_rn(-lp, sd.kdir[c], ext[c]);
  }
}

__device__ __forceinline__ void accel_add_kick(const SpeciesDev& sd, const double z[3], double ext[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) ext[c] = __fma_rn(sd.sigma, z[c], ext[c]);
}

template <bool F64>
__device__ __forceinline__ void accel_ext(const TrapDev& tp, const SpeciesDev& sd, const double k[3],
                                          const double xf[3], const double vd[3], long long counter, long long id,
                                          double ext[3]) {
  accel_ext_det(sd, k, xf, vd, ext);
  if (sd.sigma > 0.0) {
    double z[3];
    if constexpr (F64) {
      normals3_f64(tp.seed, counter, id, z);
    } else {
      float zf[3];
      normals3_f32(tp.seed, counter, id, zf);
      z[0] = zf[0], z[1] = zf[1], z[2] = zf[2];
    }
    accel_add_kick(sd, z, ext);
  }
}

__device__ __forceinline__ void accel_total(const SpeciesDev& sd, const double S[3], const double ext[3],
                                            double acc[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) acc[c] = __fma_rn(sd.coul, S[c], ext[c]);
}

// The rest of the step once the acceleration is known: v_{n+1}, the next positions and
// their pair-stream entry, the stores and the finiteness check.
__device__ __forceinline__ bool verlet_finish(const TrapDev& tp, const double xf[3], const double vd[3],
                                              const double acc[3], double vn[3], double xn[3]) {
  bool finite = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vn[c] = half_kick(vd[c], acc[c], tp.hdt);
    xn[c] = drift(xf[c], half_kick(vn[c], acc[c], tp.hdt), tp.dt);
    finite = finite && isfinite(acc[c]) && isfinite(vn[c]) && isfinite(xn[c]);
  }
  return finite;
}

// Fused epilogue for ion i: Coulomb sum S -> acceleration -> Verlet update -> next
// pair-stream entry.  cosv = cos(Omega t) at the force time.  F64 selects the plain
// FP64 form (FP64 noise, double4_32a pair stream).
template <bool F64>
__device__ __forceinline__ void epilogue_ion(const StepArgs& A, long long i, const double S[3],
                                             const double (*springs)[3], long long ns, int wb) {
  const long long n = A.n;
  const int spi = A.sp[i];
  const SpeciesDev sd = A.spc[spi];
  if (A.mode == MODE_FORCES) {
#pragma unroll
    for (int c = 0; c < 3; ++c) A.out[c * n + i] = sd.coul * S[c];
    return;
  }
  const TrapDev& tp = A.trap;
  const bool step = (A.mode == MODE_STEP);
  double xf[3], vd[3], v0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double x = A.x[c * n + i], v = A.v[c * n + i], a = A.a[c * n + i];
    const double vh = half_kick(v, a, tp.hdt);
    v0[c] = v;
    vd[c] = step ? vh : v;
    xf[c] = step ? drift(x, vh, tp.dt) : x;
  }
  double ext[3], acc[3];
  accel_ext<F64>(tp, sd, springs[spi], xf, vd, step ? ns + 1 : ns, i, ext);
  accel_total(sd, S, ext, acc);
  double vn[3], xn[3];
  bool finite = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vn[c] = step ? half_kick(vd[c], acc[c], tp.hdt) : v0[c];
    xn[c] = drift(xf[c], half_kick(vn[c], acc[c], tp.hdt), tp.dt);
    finite = finite && isfinite(acc[c]) && isfinite(vn[c]) && isfinite(xn[c]);
    if (step) {
      A.x[c * n + i] = xf[c];
      A.v[c * n + i] = vn[c];
    }
    A.a[c * n + i] = acc[c];
  }
  write_pair<F64>(A, wb, i, xn, sd.w);
  if (!finite) atomicOr(A.err, ERR_NONFINITE);
}

}  // namespace it
