// iontrap_api.cu -- host side of libiontrap.so: the C ABI declared in include/iontrap.h.
//
// A handle holds one simulation resident on the device: FP64 state (x, v, a), the
// species table, two ping-pong pair streams (FP32 hi/lo float4 or FP64 double4_32a), the
// split partials and counters the force kernel uses, and a device step counter.  Steps
// are enqueued as an instantiated CUDA graph of 100 chained kernel nodes (built node by
// node, so any stream works, including the legacy default stream) plus single launches
// for the remainder; no host round trip happens between steps.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <limits>
#include <vector>

#include "iontrap_internal.cuh"

namespace it {
// batched.cu
int batched_max_n();
bool batched_shape_fits(long long n, int C, int NP);
cudaError_t launch_batched(const std::vector<BatchEns>& ens, const std::vector<long long>& steps, int K,
                           cudaStream_t stream);
const void* step_kernel(int f64, int T, int I, int packed, int fused);
const void* epilogue_kernel(int f64);
cudaError_t allow_large_clusters();
const void* prep_kernel();
const void* restore_kernel();
cudaError_t launch_normals(unsigned long long seed, long long counter, const long long* d_ids, long long m,
                           int f64, double* d_z, cudaStream_t st);
// persistent.cu
cudaError_t launch_min_iteration(const StepArgs& s, const double* coul, void* scratch, double dt, double dmax,
                                 double ftol, int f64, int b, cudaStream_t st);
size_t min_scratch_bytes(long long n);
size_t min_state_bytes();
void min_progress(const void* host_state, long long* iters, double* fnorm, int* converged);
cudaError_t launch_hessian(const StepArgs& s, double* d_H, cudaStream_t st);
cudaError_t launch_snapshot(long long n, const double* x, const double* v, const double* a, double* snap, double dt,
                            cudaStream_t st);
cudaError_t launch_record(long long n, const double* x, const double* v, const double* a, const double* snap,
                          double* out, unsigned fields, long long W, double dt, cudaStream_t st);
cudaError_t launch_gp(const StepArgs& a, unsigned* sync, int W, int S, int G, int Lmax, long long K,
                      cudaStream_t st);
int gp_max_ctas(int W, int S, int Lmax, int max_lmax, long long max_k, int sms);
size_t rp_scratch_bytes(int NP, int JP);
cudaError_t launch_rp(const StepArgs& a, unsigned* sync, int W, int R, int NP, int JP, int I, int G, long long K,
                      cudaStream_t st);
int rp_max_ctas(int W, int R, int NP, int JP, int I, long long max_k, int sms);
size_t rp_smem_bytes(int W, int R, int NP, int JP, long long K);
}  // namespace it

using namespace it;

static constexpr int kGraphSteps = 100;
static constexpr int kMaxJsplitF64 = 2048;  // FP64 form stages its whole j-range
static constexpr int64_t kMaxSplitsUnfused = 64;
static constexpr int64_t kMaxClusterSplits = 8;   // portable cluster size (form 2)
static constexpr int64_t kMaxClusterSplits3 = 16; // non-portable cluster size (form 3)
// grid-persistent form (fused = 4)
static constexpr int64_t kGpMaxSteps = 1000;   // steps per cooperative launch
static constexpr int64_t kGpMaxSeg = 4096;     // j-segment entries staged in shared memory (128 KB)
static constexpr int64_t kGpMaxGroups = 255;   // i-groups (one counter each)
static constexpr size_t kGpSyncBytes = 32 * (1 + kGpMaxGroups) * sizeof(unsigned);

// Launch shape of the grid-persistent form: W warps per CTA, S j-segments (CTAs per
// i-group of 64 W ions), G = groups x S co-resident CTAs, Lmax entries per segment.
struct GpShape {
  int W = 0, S = 0, G = 0, Lmax = 0;
};

// row-persistent form (fused = 5): W warps, R ions per CTA, G CTAs, NP j-parts of JP entries
struct RpShape {
  int W = 0, R = 0, G = 0, NP = 0, JP = 0;
  int I = 1;  // ions per thread
};
static constexpr int64_t kRpInitJsplit = 512;  // j-range per CTA of its creation-time / force evaluation

struct iontrap {
  int64_t n = 0;
  int nspecies = 0;
  iontrap_species species[IONTRAP_MAX_SPECIES]{};
  iontrap_params p{};
  // pseudopotential trap given by per-species secular angular frequencies (rad/s), used
  // instead of Eq. 2 when pseudo_given (IONTRAP_PSEUDO only)
  double pseudo_w[IONTRAP_MAX_SPECIES][3]{};
  int pseudo_given = 0;
  iontrap_cooling cooling[IONTRAP_MAX_SPECIES]{};  // per-species cooling set by iontrap_set_params
  int cooling_given = 0;
  int f64 = 0;
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap = nullptr;  // private stream used only to capture the step graph
  // device buffers
  double *d_x = nullptr, *d_v = nullptr, *d_a = nullptr, *d_out = nullptr;
  unsigned char* d_sp = nullptr;
  void* d_pair[2] = {nullptr, nullptr};
  void* d_part = nullptr;
  size_t part_bytes = 0;
  unsigned* d_cnt = nullptr;
  size_t cnt_len = 0;
  unsigned* d_done = nullptr;
  long long* d_step = nullptr;
  int* d_err = nullptr;
  // launch configuration
  int T = 128, I = 1, packed = 0, jsplit = 128, fused = 1, pdl = 0, use_graph = 1;
  GpShape gp{};                 // fused = 4
  RpShape rp{};                 // fused = 5
  unsigned* d_gsync = nullptr;  // fused = 4, 5: step and group counters (zero between launches)
  double* d_snap = nullptr;     // iontrap_step_record: x_{s-W}, x_{s-W+1} [2][3][n]
  StepArgs args{};
  // graph of kGraphSteps chained steps
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t step = 0;  // state step index after all enqueued work
  int status = IONTRAP_OK;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Shape of a grid-persistent configuration (FP32 form with the pair term, 256 or 512
// threads, two ions per lane packed, at least seven segments, every CTA co-resident),
// or false when the configuration does not qualify.
bool gp_shape(int64_t n, int f64, unsigned flags, int sms, int T, int I, int packed, int64_t jsplit, GpShape* out) {
  if (f64 || (flags & IONTRAP_COULOMB_OFF) || (T != 256 && T != 512) || I != 2 || packed != 1 || jsplit < 1 ||
      jsplit > n)
    return false;
  const int W = T / 32;
  const int64_t S = cdiv(n, jsplit), groups = cdiv(n, 64 * (int64_t)W), Lmax = cdiv(n, S);
  // every CTA integrates at most ceil(64 W / S) ions, one thread per component
  if (S < 2 || 3 * cdiv(64 * W, S) > 32 * W || groups > kGpMaxGroups || Lmax > kGpMaxSeg) return false;
  if (S > 64 * W || groups * S > gp_max_ctas(W, (int)S, (int)Lmax, (int)kGpMaxSeg, kGpMaxSteps, sms)) return false;
  out->W = W, out->S = (int)S, out->G = (int)(groups * S), out->Lmax = (int)Lmax;
  return true;
}

double effective_dt(const iontrap_params* p) {
  if (p->dt > 0) return p->dt;
  return 2.0 * kPi / p->Omega / 20.0;
}

// ------------------------------------------------------------------ stability
// Spring constant along x (sgn = -1) or y (sgn = +1) for a species with ratio rho.
struct Spring {
  double q4, rho, a, q, wz2, Omega;
  int sgn;
  bool rf;
  double operator()(double t) const {
    const double c = rf ? std::cos(Omega * t) : 0.0;
    return q4 * rho * (a + sgn * 2.0 * q * c) - 0.5 * rho * wz2;
  }
};

// Trace of the one-period monodromy of the kick-drift-kick map of x'' = -k(t) x.
double kdk_trace(const Spring& k, double dt, int steps) {
  double m00 = 1, m01 = 0, m10 = 0, m11 = 1;
  for (int s = 0; s < steps; ++s) {
    const double k0 = k(s * dt), k1 = k((s + 1) * dt);
    const double a00 = 1 - 0.5 * dt * dt * k0, a01 = dt;
    const double a10 = -0.5 * dt * (k0 + k1) + 0.25 * dt * dt * dt * k0 * k1, a11 = 1 - 0.5 * dt * dt * k1;
    const double n00 = a00 * m00 + a01 * m10, n01 = a00 * m01 + a01 * m11;
    const double n10 = a10 * m00 + a11 * m10, n11 = a10 * m01 + a11 * m11;
    m00 = n00, m01 = n01, m10 = n10, m11 = n11;
  }
  return m00 + m11;
}

// Trace of the continuous monodromy over one RF period (RK4, 4096 substeps); used
// when dt does not divide the RF period.
double mathieu_trace(const Spring& k, double T) {
  const int sub = 4096;
  const double h = T / sub;
  double Y[2][2] = {{1, 0}, {0, 1}};
  for (int s = 0; s < sub; ++s) {
    const double t = s * h;
    for (int col = 0; col < 2; ++col) {
      const double y0 = Y[0][col], y1 = Y[1][col];
      const double k1a = y1, k1b = -k(t) * y0;
      const double k2a = y1 + h / 2 * k1b, k2b = -k(t + h / 2) * (y0 + h / 2 * k1a);
      const double k3a = y1 + h / 2 * k2b, k3b = -k(t + h / 2) * (y0 + h / 2 * k2a);
      const double k4a = y1 + h * k3b, k4b = -k(t + h) * (y0 + h * k3a);
      Y[0][col] = y0 + h / 6 * (k1a + 2 * k2a + 2 * k3a + k4a);
      Y[1][col] = y1 + h / 6 * (k1b + 2 * k2b + 2 * k3b + k4b);
    }
  }
  return Y[0][0] + Y[1][1];
}

int check_params(const iontrap_species* sp, int ns, const iontrap_params* p) {
  if (!sp || !p || ns < 1 || ns > IONTRAP_MAX_SPECIES) return IONTRAP_EINVAL;
  for (int s = 0; s < ns; ++s)
    if (!(sp[s].mass_amu > 0) || !std::isfinite(sp[s].mass_amu) || !std::isfinite(sp[s].charge_e))
      return IONTRAP_EINVAL;
  if (sp[0].charge_e == 0.0) return IONTRAP_EINVAL;  // species 0 is the a/q reference
  const double vals[] = {p->Omega, p->a, p->q, p->omega_z, p->gamma, p->T_bath, p->dt};
  for (double v : vals)
    if (!std::isfinite(v)) return IONTRAP_EINVAL;
  if (p->gamma < 0 || p->T_bath < 0 || p->dt < 0) return IONTRAP_EINVAL;
  if (p->dt == 0 && !(p->Omega > 0)) return IONTRAP_EINVAL;
  if (!(p->flags & (IONTRAP_RF_OFF | IONTRAP_TRAP_OFF)) && !(p->Omega > 0)) return IONTRAP_EINVAL;
  if (p->precision != IONTRAP_PREC_FP32 && p->precision != IONTRAP_PREC_FP64) return IONTRAP_EINVAL;
  if (p->flags & ~(IONTRAP_RF_OFF | IONTRAP_COULOMB_OFF | IONTRAP_TRAP_OFF | IONTRAP_ALLOW_UNSTABLE | IONTRAP_PSEUDO))
    return IONTRAP_EINVAL;
  return IONTRAP_OK;
}

// Spring constants (1/s^2) of the pseudopotential of Eq. 2 for a species whose
// charge/mass is rho times that of species 0: (Omega^2/4)(a_m + q_m^2/2) along x and y
// with q_m = rho q and a_m = rho a - 2 rho omega_z^2/Omega^2 (the axial field's radial
// defocusing is Eq. 3's a_x = -a_z/2), rho omega_z^2 along z.
void pseudo_springs(const iontrap_params* p, double rho, double k[3]) {
  const double O2 = p->Omega * p->Omega;
  const double wz2 = rho * p->omega_z * p->omega_z;
  const double a_m = rho * p->a - 2.0 * wz2 / O2;
  const double q_m = rho * p->q;
  const double kr = O2 / 4.0 * (a_m + 0.5 * q_m * q_m);
  k[0] = kr;
  k[1] = kr;
  k[2] = wz2;
}

// Static springs hold an ion under kick-drift-kick when 0 < k dt^2 < 4 on every axis.
bool springs_stable(const double k[3], double dt) {
  for (int c = 0; c < 3; ++c)
    if (!(k[c] > 0.0) || !(k[c] * dt * dt < 4.0)) return false;
  return true;
}

bool species_stable(const iontrap_params* p, double rho) {
  if (p->flags & IONTRAP_TRAP_OFF) return true;
  const double dt = effective_dt(p);
  if (p->flags & IONTRAP_PSEUDO) {
    if (rho == 0.0) return true;
    double k[3];
    pseudo_springs(p, rho, k);
    return springs_stable(k, dt);
  }
  const double wz2 = rho * p->omega_z * p->omega_z;
  if (rho == 0.0) return true;  // neutral: no trap force at all
  if (!(wz2 > 0) || !(std::fabs(2.0 - dt * dt * wz2) < 2.0)) return false;
  const bool rf = !(p->flags & IONTRAP_RF_OFF);
  for (int sgn : {-1, 1}) {
    Spring k{p->Omega * p->Omega / 4.0, rho, p->a, p->q, p->omega_z * p->omega_z, p->Omega, sgn, rf};
    double tr;
    if (!rf) {
      tr = 2.0 - dt * dt * k(0.0);
    } else {
      const double Trf = 2.0 * kPi / p->Omega;
      const double K = Trf / dt;
      const double Kr = std::nearbyint(K);
      if (std::fabs(K - Kr) < 1e-9 * K && Kr >= 1 && Kr <= 100000)
        tr = kdk_trace(k, dt, (int)Kr);
      else
        tr = mathieu_trace(k, Trf);
    }
    if (!(std::fabs(tr) < 2.0)) return false;
  }
  return true;
}

// ------------------------------------------------------------------ configuration
int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// Process-wide tuning table: (device, precision, floor(log2 n)) -> configuration.
struct TuneKey {
  int dev, prec, log2n;
  bool operator<(const TuneKey& o) const {
    return dev != o.dev ? dev < o.dev : (prec != o.prec ? prec < o.prec : log2n < o.log2n);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, iontrap_tuning_entry> g_tune;

int log2_floor(int64_t n) {
  int k = 0;
  while ((n >> (k + 1)) > 0) ++k;
  return k;
}

bool tuned_config(int64_t n, int f64, int dev, iontrap_config* c) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(TuneKey{dev, f64, log2_floor(n)});
  if (it == g_tune.end()) return false;
  const iontrap_tuning_entry& e = it->second;
  c->threads = e.threads;
  c->ions_per_thread = e.ions_per_thread;
  c->packed = e.packed;
  c->fused = e.fused;
  c->pdl = e.pdl;
  c->graph = e.graph;
  c->jsplit = (int32_t)std::max<int64_t>(1, cdiv(n, std::max(1, e.splits)));
  return true;
}

// Default tile configuration for n ions.  The i-block (T*I ions) grows with n: small
// blocks keep the FP64 epilogue of the last CTA short, large ones reuse each staged j
// over more ions.  The number of j-splits S makes the grid a multiple of the SM count
// (equal work per SM) with at least two CTAs per SM where n allows.
// Row-persistent shape: R ions per CTA (3 R threads integrate, so R <= 32 W / 3), NP =
// 32 W / R j-parts per CTA, JP entries per part: a multiple of 4 (16-byte shared loads of
// four j, 16-byte aligned arrays), with JP / 4 odd when a warp spans several parts (R not
// a multiple of 32), so that their loads start in distinct banks; the launch must fit in
// shared memory and on the GPU at once.
// With two ions per thread (I = 2) the parts are NP = 32 W / ceil(R / 2).
bool rp_shape(int64_t n, int f64, unsigned flags, int sms, int T, int I, int packed, int64_t R, RpShape* out) {
  if (f64 || (flags & IONTRAP_COULOMB_OFF) || (T != 256 && T != 512) || (I != 1 && I != 2) || packed != 1 || R < 1 ||
      R > n)
    return false;
  const int W = T / 32;
  if (3 * R > 32 * W) return false;
  const int64_t RT = cdiv(R, I);
  const int64_t NP = (32 * W) / RT;
  int64_t q4 = cdiv(cdiv(n, NP), 4);
  if (RT % 32 != 0 && !(q4 & 1)) ++q4;
  const int64_t JP = 4 * q4, G = cdiv(n, R);
  if (rp_smem_bytes(W, (int)R, (int)NP, (int)JP, kGpMaxSteps) > 227 * 1024) return false;
  if (G > rp_max_ctas(W, (int)R, (int)NP, (int)JP, I, kGpMaxSteps, sms)) return false;
  out->W = W, out->R = (int)R, out->G = (int)G, out->NP = (int)NP, out->JP = (int)JP, out->I = I;
  return true;
}

void default_config(int64_t n, int f64, int sms, int* T, int* I, int* packed, int* jsplit, int* fused,
                    int allow_persistent = 1) {
  *fused = 1;
  if (f64) {
    *T = 128;
    *I = 1;
    *packed = 0;
  } else if (n <= 8192) {
    *T = 64, *I = 1, *packed = 0;
  } else if (n <= 32768) {
    *T = 128, *I = 4, *packed = 1;
  } else {
    *T = 128, *I = 4, *packed = 1;
  }
  // Split count S: a score of wave efficiency (CTAs fill whole waves of SMs), fill (at
  // least two CTAs per SM) and a small preference for fewer splits (less partial
  // traffic); at most 64 splits, at least 32 j per split.
  const int64_t iblocks = cdiv(n, (int64_t)(*T) * (*I));
  // (the FP64 form, whose pair term runs at the FP64 rate, spreads small n more thinly:
  // at least 8 j per split instead of 32)
  const int64_t s_max = std::max<int64_t>(1, std::min<int64_t>(64, n / (f64 ? 8 : 32)));
  int64_t S = 1;
  double best = -1e30;
  for (int64_t cand = 1; cand <= s_max; ++cand) {
    const double ctas = (double)(iblocks * cand);
    const double waves = ctas / sms;
    const double eff = waves / std::ceil(waves);
    const double fill = std::min(1.0, ctas / (2.0 * sms));
    const double score = eff * fill - 0.002 * (double)cand;
    if (score > best + 1e-12) {
      best = score;
      S = cand;
    }
  }
  // the FP64 form at small n: every split it may take (its pair term is latency-bound on
  // few SMs; n = 64: 8 CTAs of 8 j instead of one)
  if (f64 && iblocks * s_max <= sms) S = s_max;
  int64_t js = cdiv(n, S);
  if (f64) js = std::min<int64_t>(js, kMaxJsplitF64);
  if (!*fused && cdiv(n, js) > kMaxSplitsUnfused) js = cdiv(n, kMaxSplitsUnfused);
  *jsplit = (int)js;
  // 2048 < n <= 8192: the cluster + warp-split form (4 warps, 2 ions per lane, 8-CTA
  // clusters) measured fastest (20.8 us/step at n = 4096 against 24.7 for the others)
  if (!f64 && n > 2048 && n <= 8192) {
    *T = 128, *I = 2, *packed = 1, *fused = 3;
    *jsplit = (int)cdiv(n, 8);
  }
  // 2048 <= n <= 8192: the grid-persistent form with one CTA per SM measured faster
  // still (n = 2048: 9.5 against 17.0 us/step; 4096: 17.6 against 20.4; 8192: 50.6
  // against 52.5); callers that overlap many simulations opt out with allow_persistent = 0
  if (!f64 && allow_persistent && n >= 2048 && n <= 8192) {
    const int W = n <= 2048 ? 8 : 16;
    const int64_t S = sms / cdiv(n, 64 * (int64_t)W);
    GpShape gs;
    if (S >= 7 && gp_shape(n, 0, 0, sms, 32 * W, 2, 1, cdiv(n, S), &gs)) {
      *T = 32 * W, *I = 2, *packed = 1, *fused = 4;
      *jsplit = (int)cdiv(n, S);
    }
  }
  // Wherever its staged j fit in shared memory (n up to about 7000): the row-persistent
  // form with the ions spread over every SM measured fastest of all (us/step on GB300
  // against the choices above: n = 1024: 5.3 vs 13.4; 2048: 6.7 vs 9.7; 3000: 9.7 vs 13.0;
  // 4096: 14.6 vs 17.3; 6000: 25.9 vs 30.6).  Ions per CTA: of ceil(n / SMs) and the next
  // three counts, the one with the shortest j-part (the pair loop's length), then the
  // most threads in the loop (n = 4096: 28 ions, 18 parts of 228 j and 504 busy threads,
  // measured 12.9 against 13.3 us/step for 27 ions and 486 threads)
  if (!f64 && allow_persistent) {
    const int W = n < 2048 ? 8 : 16;
    RpShape best{};
    bool found = false;
    for (int64_t R = cdiv(n, sms); R < cdiv(n, sms) + 4; ++R) {
      RpShape rs;
      if (!rp_shape(n, 0, 0, sms, 32 * W, 1, 1, R, &rs)) continue;
      if (!found || rs.JP < best.JP || (rs.JP == best.JP && rs.R * rs.NP > best.R * best.NP)) best = rs;
      found = true;
    }
    if (found) {
      *T = 32 * W, *I = 1, *packed = 1, *fused = 5;
      *jsplit = best.R;
    }
    // up to 112 ions: all of them in one CTA of 16 warps, whose pair work costs less than
    // a grid-wide barrier between steps (us/step, one CTA against the ions spread over
    // every SM: n = 16: 2.8 vs 5.7; 64: 3.3 vs 5.7; 100: 5.0 vs 5.8; 128: 5.8 vs 5.8)
    RpShape one;
    if (n <= 112 && rp_shape(n, 0, 0, sms, 512, 1, 1, n, &one)) {
      *T = 512, *I = 1, *packed = 1, *fused = 5;
      *jsplit = (int)n;
    }
  }
}

int set_status(iontrap* h, int st) {
  if (st != IONTRAP_OK && h->status == IONTRAP_OK) h->status = st;
  return h->status;
}

int cuda_status(iontrap* h, cudaError_t e) {
  if (e == cudaSuccess) return h->status;
  return set_status(h, e == cudaErrorMemoryAllocation ? IONTRAP_ENOMEM : IONTRAP_ECUDA);
}

int64_t splits_of(const iontrap* h) {
  if (h->p.flags & IONTRAP_COULOMB_OFF) return 1;
  if (h->fused == 5) return cdiv(h->n, kRpInitJsplit);
  return cdiv(h->n, h->jsplit);
}

// ions per i-block: T*I, except the cluster + warp-split form (fused = 3) whose warps
// all hold the same 32*I ions, and the grid-persistent form (fused = 4) whose initial
// evaluation at creation uses the last-CTA form with 128 x 2 ions
int64_t iblock_ions(const iontrap* h) {
  if (h->fused >= 4) return 256;
  return h->fused == 3 ? 32 * (int64_t)h->I : (int64_t)h->T * h->I;
}

dim3 grid_of(const iontrap* h) {
  return dim3((unsigned)cdiv(h->n, iblock_ions(h)), (unsigned)splits_of(h), 1);
}

size_t smem_of(const iontrap* h) {
  if (!h->f64 || (h->p.flags & IONTRAP_COULOMB_OFF)) return 0;  // FP32 form: static chunk buffers
  return (size_t)h->jsplit * 32;
}

// The per-species constants and the trap of a handle's step arguments, from the trap and
// default bath of p and, when cool is not null, one bath and laser per species.
void fill_forces(iontrap* h, const iontrap_params* p, const iontrap_cooling* cool) {
  const double dt = h->p.dt;
  const double ke = 1.0 / (4.0 * kPi * kEps0);
  const double qm0 = h->species[0].charge_e / h->species[0].mass_amu;
  StepArgs& A = h->args;
  int laser = 0;
  for (int s = 0; s < h->nspecies; ++s) {
    const double M = h->species[s].mass_amu * kAmu, z = h->species[s].charge_e;
    const double g = cool ? cool[s].gamma : p->gamma, T = cool ? cool[s].T_bath : p->T_bath;
    SpeciesDev& d = A.spc[s];
    d.coul = ke * kE * kE * z / M;
    d.rho = (z / h->species[s].mass_amu) / qm0;
    d.gamma = g;
    d.sigma = std::sqrt(2.0 * g * kKB * T / (M * dt));
    const double* L = cool ? cool[s].laser : nullptr;
    const double ln = L ? std::sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]) : 0.0;
    d.lrate = ln;
    for (int c = 0; c < 3; ++c) d.kdir[c] = ln > 0.0 ? L[c] / ln : 0.0;
    if (ln > 0.0) laser = 1;
    if (h->pseudo_given) {
      for (int c = 0; c < 3; ++c) d.ks[c] = h->pseudo_w[s][c] * h->pseudo_w[s][c];
    } else {
      pseudo_springs(p, d.rho, d.ks);
    }
    d.mass = M;
    d.z = z;
    d.w = (float)z;
    d.pad = 0.f;
  }
  A.trap.dt = dt;
  A.trap.hdt = 0.5 * dt;
  A.trap.Omega = p->Omega;
  A.trap.q4 = p->Omega * p->Omega / 4.0;
  A.trap.a = p->a;
  A.trap.q = p->q;
  A.trap.wz2 = p->omega_z * p->omega_z;
  A.trap.seed = p->seed;
  A.trap.flags = p->flags;
  A.trap.laser = laser;
}

void destroy_graph(iontrap* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
}

// Device buffers of a handle come from a per-device pool of the stream-ordered allocator
// and are allocated and freed in order on the handle's stream: unlike cudaMalloc and
// cudaFree neither synchronises the device, so a handle created or destroyed while others
// run (the serving loop admits and retires requests between their chunks) does not stall
// them.  The pool keeps up to kPoolKeepBytes of freed memory for reuse.
constexpr uint64_t kPoolKeepBytes = (uint64_t)4 << 30;

cudaMemPool_t handle_pool(int dev) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lock(mu);
  auto f = pools.find(dev);
  if (f != pools.end()) return f->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
  uint64_t keep = kPoolKeepBytes;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = pool;
  return pool;
}

template <typename T>
cudaError_t dev_alloc(const iontrap* h, T** p, size_t bytes) {
  cudaMemPool_t pool = handle_pool(h->device);
  if (!pool) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes, pool, h->stream);
}

void dev_free(const iontrap* h, void* p) {
  if (p) cudaFreeAsync(p, h->stream);
}

// (Re)allocate the scratch that depends on the tile configuration.
int alloc_scratch(iontrap* h) {
  const int64_t splits = splits_of(h);
  if (h->fused == 5 &&
      !rp_shape(h->n, h->f64, h->p.flags, h->sms, h->T, h->I, h->packed, h->jsplit, &h->rp))
    return IONTRAP_EINVAL;
  // one 32-byte record per (split, ion) in both forms; the row-persistent form also keeps
  // its part-major position copies there between the steps of a launch
  size_t part = (size_t)splits * (size_t)h->n * 32;
  if (h->fused == 5) part = std::max(part, rp_scratch_bytes(h->rp.NP, h->rp.JP));
  const size_t cnt = (size_t)cdiv(h->n, iblock_ions(h));
  if (part > h->part_bytes) {
    dev_free(h, h->d_part);
    h->d_part = nullptr;
    h->part_bytes = 0;
    if (dev_alloc(h, &h->d_part, part) != cudaSuccess) return IONTRAP_ENOMEM;
    h->part_bytes = part;
  }
  if (cnt > h->cnt_len) {
    dev_free(h, h->d_cnt);
    h->d_cnt = nullptr;
    h->cnt_len = 0;
    if (dev_alloc(h, &h->d_cnt, cnt * sizeof(unsigned)) != cudaSuccess) return IONTRAP_ENOMEM;
    h->cnt_len = cnt;
  }
  if (cudaMemsetAsync(h->d_cnt, 0, h->cnt_len * sizeof(unsigned), h->stream) != cudaSuccess)
    return IONTRAP_ECUDA;
  if (h->fused == 4 || h->fused == 5) {
    if (h->fused == 4 &&
        !gp_shape(h->n, h->f64, h->p.flags, h->sms, h->T, h->I, h->packed, h->jsplit, &h->gp))
      return IONTRAP_EINVAL;
    if (!h->d_gsync) {
      if (dev_alloc(h, &h->d_gsync, kGpSyncBytes) != cudaSuccess) return IONTRAP_ENOMEM;
      if (cudaMemsetAsync(h->d_gsync, 0, kGpSyncBytes, h->stream) != cudaSuccess) return IONTRAP_ECUDA;
    }
  }
  h->args.part = h->d_part;
  h->args.cnt = h->d_cnt;
  h->args.jsplit = (h->p.flags & IONTRAP_COULOMB_OFF) ? (int)std::min<int64_t>(h->n, 1 << 30)
                   : h->fused == 5                   ? (int)std::min<int64_t>(h->n, kRpInitJsplit)
                                                     : h->jsplit;
  h->args.nsplit = (int)splits;
  return IONTRAP_OK;
}

// One row-persistent launch of K steps on the handle's buffers.
cudaError_t launch_rp_of(iontrap* h, const StepArgs& a, long long K, cudaStream_t st) {
  return launch_rp(a, h->d_gsync, h->rp.W, h->rp.R, h->rp.NP, h->rp.JP, h->rp.I, h->rp.G, K, st);
}

// Launch one step kernel with programmatic dependent launch, so that consecutive steps
// overlap one grid's launch with the previous grid's tail.
cudaError_t launch_step_on(iontrap* h, StepArgs& a, cudaStream_t st) {
  if (h->fused == 5 && a.mode != MODE_INIT)
    return launch_rp_of(h, a, 1, st);
  if (h->fused == 4 || h->fused == 5) {
    if (h->fused == 4 && a.mode != MODE_INIT)
      return launch_gp(a, h->d_gsync, h->gp.W, h->gp.S, h->gp.G, h->gp.Lmax, 1, st);
    // the initial evaluation (at creation or after restore): the last-CTA form over the same j-segments
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)cdiv(h->n, 256), (unsigned)splits_of(h), 1);
    cfg.blockDim = dim3(128);
    cfg.stream = st;
    void* params[] = {&a};
    return cudaLaunchKernelExC(&cfg, step_kernel(0, 128, 2, 1, 1), params);
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid_of(h);
  cfg.blockDim = dim3(h->T);
  cfg.dynamicSmemBytes = smem_of(h);
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (h->pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (h->fused >= 2) {  // the j-splits of an i-block form one cluster
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = 1;
    attr[na].val.clusterDim.y = cfg.gridDim.y;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  void* params[] = {&a};
  cudaError_t e = cudaLaunchKernelExC(&cfg, step_kernel(h->f64, h->T, h->I, h->packed, h->fused), params);
  if (e != cudaSuccess || h->fused != 0) return e;
  cfg.gridDim = dim3((unsigned)cdiv(h->n, 32));  // 32 ions per epilogue CTA
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  return cudaLaunchKernelExC(&cfg, epilogue_kernel(h->f64), params);
}

cudaError_t launch_mode(iontrap* h, int mode, double* out) {
  StepArgs a = h->args;
  a.mode = mode;
  a.out = out;
  return launch_step_on(h, a, h->stream);
}

cudaError_t launch_prep(iontrap* h, int b) {
  int f64 = h->f64;
  void* params[] = {&h->args, &b, &f64};
  const unsigned blocks = (unsigned)std::min<int64_t>(cdiv(h->n, 256), 4096);
  return cudaLaunchKernel(prep_kernel(), dim3(blocks), dim3(256), params, 0, h->stream);
}

cudaError_t launch_restore(iontrap* h, int b) {
  int f64 = h->f64;
  void* params[] = {&h->args, &b, &f64};
  const unsigned blocks = (unsigned)std::min<int64_t>(cdiv(h->n, 256), 4096);
  return cudaLaunchKernel(restore_kernel(), dim3(blocks), dim3(256), params, 0, h->stream);
}

// Capture kGraphSteps chained PDL step launches on the private capture stream; the
// instantiated graph is then launched on the handle's stream (any stream works).
cudaError_t build_graph(iontrap* h) {
  destroy_graph(h);
  if (!h->cap) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  StepArgs a = h->args;
  a.mode = MODE_STEP;
  a.out = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int s = 0; s < kGraphSteps && e == cudaSuccess; ++s) e = launch_step_on(h, a, h->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e;
  }
  h->graph = g;
  return cudaGraphInstantiate(&h->gexec, h->graph, 0);
}

int prepare_kernels() {
  static int done = 0;
  if (done) return IONTRAP_OK;
  const int Ts[] = {64, 128, 256};
  const int Is[] = {1, 2, 4};
  for (int T : Ts)
    for (int I : Is) {
      const void* fn = step_kernel(1, T, I, 0, 1);
      if (fn && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxJsplitF64 * 32) !=
                    cudaSuccess)
        return IONTRAP_ECUDA;
    }
  if (allow_large_clusters() != cudaSuccess) return IONTRAP_ECUDA;
  done = 1;
  return IONTRAP_OK;
}

// a_n again under the handle's current forces at its current state (as creation does).
int reevaluate(iontrap* h) {
  cudaError_t e = launch_prep(h, (int)(h->step & 1));
  if (e == cudaSuccess) e = launch_mode(h, MODE_INIT, nullptr);
  if (e != cudaSuccess) return cuda_status(h, e);
  return iontrap_sync(h);
}

void free_all(iontrap* h) {
  destroy_graph(h);
  void* ptrs[] = {h->d_x, h->d_v, h->d_a, h->d_out, h->d_sp, h->d_pair[0], h->d_pair[1],
                  h->d_part, h->d_cnt, h->d_done, h->d_step, h->d_err, h->d_gsync, h->d_snap};
  for (void* q : ptrs) dev_free(h, q);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  if (h->cap) cudaStreamDestroy(h->cap);
}

}  // namespace

namespace it {
// The batched launch's group shape for ensembles of n ions on device dev, if tuned: CTAs
// per group and j-parts (0: the launcher's cost model).
bool batched_tuned_shape(int dev, long long n, int* C, int* NP) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto f = g_tune.find(TuneKey{dev, IONTRAP_TUNE_BATCHED, log2_floor(n)});
  if (f == g_tune.end()) return false;
  *C = f->second.splits;
  *NP = f->second.ions_per_thread;
  return true;
}

// Move an idle handle that does not own its stream onto another stream of its device; its
// later work (and the release of its buffers) is enqueued there.  The serving loop
// creates handles on a private stream, so that admission never waits for a chunk in
// flight, and then steps them on shared ones.
int rebind_stream(iontrap* h, cudaStream_t st) {
  if (!h || !st || h->own_stream) return IONTRAP_EINVAL;
  h->stream = st;
  return IONTRAP_OK;
}

// Give a handle the default configuration without the grid-persistent form (for callers
// that run many simulations side by side on separate streams).
int use_nonpersistent_default(iontrap* h) {
  if (!h || h->fused < 4) return IONTRAP_OK;
  iontrap_config c{};
  const int st = iontrap_default_config(h->n, h->f64 ? IONTRAP_PREC_FP64 : IONTRAP_PREC_FP32, h->p.flags, 0, &c);
  return st ? st : iontrap_set_config(h, &c);
}
}  // namespace it

// ==================================================================== C ABI
extern "C" {

const char* iontrap_strerror(int status) {
  switch (status) {
    case IONTRAP_OK: return "ok";
    case IONTRAP_EINVAL: return "invalid argument";
    case IONTRAP_ENOMEM: return "device memory allocation failed";
    case IONTRAP_EUNSTABLE: return "trap parameters give unbounded single-ion motion for a species";
    case IONTRAP_ENONFINITE: return "a step produced a non-finite acceleration, velocity or position";
    case IONTRAP_ETIMEOUT: return "a bounded device-side wait expired";
    case IONTRAP_ECUDA: return "CUDA runtime error";
    case IONTRAP_ETOOLARGE: return "n exceeds the allocation-free scratch capacity (8192 ions)";
    default: return "unknown status";
  }
}

int iontrap_linear_pt(double V0, double U0, double R0, double Z0, double kappa, double Omega,
                      const iontrap_species* species0, iontrap_params* p) {
  if (!species0 || !p) return IONTRAP_EINVAL;
  const double vals[] = {V0, U0, R0, Z0, kappa, Omega, species0->mass_amu, species0->charge_e};
  for (double v : vals)
    if (!std::isfinite(v)) return IONTRAP_EINVAL;
  if (!(R0 > 0) || !(Z0 > 0) || !(Omega > 0) || !(species0->mass_amu > 0)) return IONTRAP_EINVAL;
  const double qm = species0->charge_e * kE / (species0->mass_amu * kAmu);  // Q/M, C/kg
  const double wz2 = 2.0 * qm * kappa * U0 / (Z0 * Z0);
  if (wz2 < 0) return IONTRAP_EINVAL;
  p->Omega = Omega;
  p->a = 0.0;
  p->q = 2.0 * qm * V0 / (R0 * R0 * Omega * Omega);
  p->omega_z = std::sqrt(wz2);
  return IONTRAP_OK;
}

int iontrap_stable(const iontrap_species* species, int n_species, const iontrap_params* p, int* is_stable) {
  if (!is_stable) return IONTRAP_EINVAL;
  const int st = check_params(species, n_species, p);
  if (st) return st;
  const double qm0 = species[0].charge_e / species[0].mass_amu;
  int ok = 1;
  for (int s = 0; s < n_species && ok; ++s)
    ok = species_stable(p, (species[s].charge_e / species[s].mass_amu) / qm0) ? 1 : 0;
  *is_stable = ok;
  return IONTRAP_OK;
}

int iontrap_create(const iontrap_species* species, int n_species, const uint8_t* species_of_ion,
                   const double* x0, const double* v0, int64_t n, const iontrap_params* p, int64_t step0,
                   void* cuda_stream, iontrap_t** out) {
  if (!out) return IONTRAP_EINVAL;
  *out = nullptr;
  if (n < 1 || !species_of_ion || !x0 || step0 < 0) return IONTRAP_EINVAL;
  int st = check_params(species, n_species, p);
  if (st) return st;
  for (int64_t i = 0; i < n; ++i)
    if (species_of_ion[i] >= n_species) return IONTRAP_EINVAL;
  for (int64_t k = 0; k < 3 * n; ++k)
    if (!std::isfinite(x0[k]) || (v0 && !std::isfinite(v0[k]))) return IONTRAP_EINVAL;
  if (!(p->flags & IONTRAP_ALLOW_UNSTABLE)) {
    int ok = 0;
    iontrap_stable(species, n_species, p, &ok);
    if (!ok) return IONTRAP_EUNSTABLE;
  }

  iontrap* h = new (std::nothrow) iontrap();
  if (!h) return IONTRAP_ENOMEM;
  h->n = n;
  h->nspecies = n_species;
  h->p = *p;
  h->p.dt = effective_dt(p);
  h->f64 = p->precision == IONTRAP_PREC_FP64;
  h->step = step0;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return IONTRAP_ECUDA;
  }
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (h->sms <= 0) h->sms = 1;
  if (prepare_kernels()) {
    delete h;
    return IONTRAP_ECUDA;
  }
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return IONTRAP_ECUDA;
    }
    h->own_stream = true;
  }
  default_config(n, h->f64, h->sms, &h->T, &h->I, &h->packed, &h->jsplit, &h->fused);
  if ((p->flags & IONTRAP_COULOMB_OFF) && h->fused >= 2) {  // cluster forms need the pair term
    h->T = 64, h->I = 1, h->packed = 0, h->fused = 1;
  }
  {
    iontrap_config tc{};
    GpShape gs;
    const bool tuned = tuned_config(n, h->f64, h->device, &tc);
    RpShape rs;
    if (tuned && tc.fused == 4) {
      if (gp_shape(n, h->f64, p->flags, h->sms, tc.threads, tc.ions_per_thread, tc.packed, tc.jsplit, &gs)) {
        h->T = tc.threads, h->I = tc.ions_per_thread, h->packed = tc.packed, h->jsplit = tc.jsplit;
        h->fused = 4, h->pdl = 0, h->use_graph = 0;
      }
    } else if (tuned && tc.fused == 5) {
      if (rp_shape(n, h->f64, p->flags, h->sms, tc.threads, tc.ions_per_thread, tc.packed, tc.jsplit, &rs)) {
        h->T = tc.threads, h->I = tc.ions_per_thread, h->packed = tc.packed, h->jsplit = tc.jsplit;
        h->fused = 5, h->pdl = 0, h->use_graph = 0;
      }
    } else if (tuned && step_kernel(h->f64, tc.threads, tc.ions_per_thread, tc.packed, tc.fused) &&
        tc.jsplit >= 1 && tc.jsplit <= n && (!h->f64 || tc.jsplit <= kMaxJsplitF64) &&
        (tc.fused || cdiv(n, tc.jsplit) <= kMaxSplitsUnfused) &&
        (tc.fused < 2 || (cdiv(n, tc.jsplit) <= (tc.fused == 3 ? kMaxClusterSplits3 : kMaxClusterSplits) &&
                          !(p->flags & IONTRAP_COULOMB_OFF)))) {
      h->T = tc.threads, h->I = tc.ions_per_thread, h->packed = tc.packed, h->jsplit = tc.jsplit;
      h->fused = tc.fused, h->pdl = tc.pdl, h->use_graph = tc.graph;
    }
  }

  // species table, trap and bath
  for (int s = 0; s < n_species; ++s) h->species[s] = species[s];
  fill_forces(h, p, nullptr);
  StepArgs& A = h->args;
  A.n = n;
  A.unitw = 1;  // every species singly charged (+1 e): exact to drop the z_j factor
  for (int s = 0; s < n_species; ++s)
    if (species[s].charge_e != 1.0) A.unitw = 0;

  const size_t vec = 3 * (size_t)n * sizeof(double);
  const size_t pair = (size_t)n * (h->f64 ? sizeof(double4_32a) : 2 * sizeof(float4));
  bool ok = dev_alloc(h, &h->d_x, vec) == cudaSuccess && dev_alloc(h, &h->d_v, vec) == cudaSuccess &&
            dev_alloc(h, &h->d_a, vec) == cudaSuccess && dev_alloc(h, &h->d_sp, (size_t)n) == cudaSuccess &&
            dev_alloc(h, &h->d_pair[0], pair) == cudaSuccess && dev_alloc(h, &h->d_pair[1], pair) == cudaSuccess &&
            dev_alloc(h, &h->d_done, sizeof(unsigned)) == cudaSuccess &&
            dev_alloc(h, &h->d_step, sizeof(long long)) == cudaSuccess &&
            dev_alloc(h, &h->d_err, sizeof(int)) == cudaSuccess;
  if (!ok) {
    free_all(h);
    delete h;
    return IONTRAP_ENOMEM;
  }
  for (int b = 0; b < 2; ++b) {
    if (h->f64) {
      A.p64[b] = (double4_32a*)h->d_pair[b];
      A.hi[b] = A.lo[b] = nullptr;
    } else {
      A.hi[b] = (float4*)h->d_pair[b];
      A.lo[b] = (float4*)h->d_pair[b] + n;
      A.p64[b] = nullptr;
    }
  }
  A.x = h->d_x;
  A.v = h->d_v;
  A.a = h->d_a;
  A.sp = h->d_sp;
  A.done = h->d_done;
  A.step = h->d_step;
  A.err = h->d_err;
  st = alloc_scratch(h);
  if (st) {
    free_all(h);
    delete h;
    return st;
  }
  long long s0 = step0;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  chk(cudaMemcpyAsync(h->d_x, x0, vec, cudaMemcpyHostToDevice, h->stream));
  if (v0)
    chk(cudaMemcpyAsync(h->d_v, v0, vec, cudaMemcpyHostToDevice, h->stream));
  else
    chk(cudaMemsetAsync(h->d_v, 0, vec, h->stream));
  chk(cudaMemcpyAsync(h->d_sp, species_of_ion, (size_t)n, cudaMemcpyHostToDevice, h->stream));
  chk(cudaMemcpyAsync(h->d_step, &s0, sizeof(s0), cudaMemcpyHostToDevice, h->stream));
  chk(cudaMemsetAsync(h->d_done, 0, sizeof(unsigned), h->stream));
  chk(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  chk(cudaMemsetAsync(h->d_a, 0, vec, h->stream));
  chk(launch_prep(h, (int)(step0 & 1)));
  chk(launch_mode(h, MODE_INIT, nullptr));
  chk(cudaStreamSynchronize(h->stream));
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? IONTRAP_ENOMEM : IONTRAP_ECUDA;
  }
  *out = h;
  return IONTRAP_OK;
}

int iontrap_step(iontrap_t* h, int64_t n_steps) {
  if (!h || n_steps < 0) return IONTRAP_EINVAL;
  if (h->status) return h->status;
  DeviceGuard g(h->device);
  if (h->fused == 4 || h->fused == 5) {  // persistent forms: up to kGpMaxSteps steps per cooperative launch
    StepArgs a = h->args;
    a.mode = MODE_STEP;
    a.out = nullptr;
    while (n_steps > 0) {
      const int64_t k = std::min<int64_t>(n_steps, kGpMaxSteps);
      cudaError_t e = h->fused == 4 ? launch_gp(a, h->d_gsync, h->gp.W, h->gp.S, h->gp.G, h->gp.Lmax, k, h->stream)
                                    : launch_rp_of(h, a, k, h->stream);
      if (e != cudaSuccess) return cuda_status(h, e);
      n_steps -= k;
      h->step += k;
    }
    return h->status;
  }
  if (n_steps >= kGraphSteps && h->use_graph && !h->gexec) {
    cudaError_t e = build_graph(h);
    if (e != cudaSuccess) return cuda_status(h, e);
  }
  while (h->use_graph && n_steps >= kGraphSteps) {
    cudaError_t e = cudaGraphLaunch(h->gexec, h->stream);
    if (e != cudaSuccess) return cuda_status(h, e);
    n_steps -= kGraphSteps;
    h->step += kGraphSteps;
  }
  for (; n_steps > 0; --n_steps) {
    cudaError_t e = launch_mode(h, MODE_STEP, nullptr);
    if (e != cudaSuccess) return cuda_status(h, e);
    h->step += 1;
  }
  return h->status;
}

int iontrap_set_params(iontrap_t* h, const iontrap_params* p, const iontrap_cooling* cooling) {
  if (!h || !p) return IONTRAP_EINVAL;
  if (h->status) return h->status;
  int st = check_params(h->species, h->nspecies, p);
  if (st) return st;
  if (effective_dt(p) != h->p.dt || p->seed != h->p.seed || p->precision != h->p.precision ||
      ((p->flags ^ h->p.flags) & IONTRAP_COULOMB_OFF))
    return IONTRAP_EINVAL;
  if (cooling)
    for (int s = 0; s < h->nspecies; ++s) {
      const iontrap_cooling& c = cooling[s];
      const double vals[] = {c.gamma, c.T_bath, c.laser[0], c.laser[1], c.laser[2]};
      for (double v : vals)
        if (!std::isfinite(v)) return IONTRAP_EINVAL;
      if (c.gamma < 0 || c.T_bath < 0) return IONTRAP_EINVAL;
    }
  if (!(p->flags & IONTRAP_ALLOW_UNSTABLE)) {
    int ok = 0;
    iontrap_stable(h->species, h->nspecies, p, &ok);
    if (!ok) return IONTRAP_EUNSTABLE;
  }
  DeviceGuard g(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);  // no graph of the old forces in flight
  if (e != cudaSuccess) return cuda_status(h, e);
  const double dt = h->p.dt;
  h->p = *p;
  h->p.dt = dt;
  h->cooling_given = cooling != nullptr;
  for (int s = 0; s < h->nspecies && cooling; ++s) h->cooling[s] = cooling[s];
  if (!(p->flags & IONTRAP_PSEUDO)) h->pseudo_given = 0;
  fill_forces(h, p, cooling);
  destroy_graph(h);
  // a_n under the new forces, as iontrap_create evaluates it at step0 = n
  return reevaluate(h);
}

int iontrap_set_pseudo_frequencies(iontrap_t* h, const double* omega) {
  if (!h) return IONTRAP_EINVAL;
  if (h->status) return h->status;
  if (!(h->p.flags & IONTRAP_PSEUDO)) return IONTRAP_EINVAL;
  if (omega) {
    for (int s = 0; s < 3 * h->nspecies; ++s)
      if (!std::isfinite(omega[s]) || !(omega[s] > 0)) return IONTRAP_EINVAL;
    if (!(h->p.flags & IONTRAP_ALLOW_UNSTABLE))
      for (int s = 0; s < h->nspecies; ++s) {
        const double k[3] = {omega[3 * s] * omega[3 * s], omega[3 * s + 1] * omega[3 * s + 1],
                             omega[3 * s + 2] * omega[3 * s + 2]};
        if (!springs_stable(k, h->p.dt)) return IONTRAP_EUNSTABLE;
      }
  } else if (!(h->p.flags & IONTRAP_ALLOW_UNSTABLE)) {
    int ok = 0;
    iontrap_stable(h->species, h->nspecies, &h->p, &ok);
    if (!ok) return IONTRAP_EUNSTABLE;
  }
  DeviceGuard g(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(h, e);
  h->pseudo_given = omega != nullptr;
  for (int s = 0; s < h->nspecies && omega; ++s)
    for (int c = 0; c < 3; ++c) h->pseudo_w[s][c] = omega[3 * s + c];
  fill_forces(h, &h->p, h->cooling_given ? h->cooling : nullptr);
  destroy_graph(h);
  return reevaluate(h);
}

int iontrap_minimize(iontrap_t* h, int64_t max_iters, double dt, double dmax, double ftol, int64_t* iters,
                     double* fnorm) {
  if (!h || max_iters < 0 || !std::isfinite(dt) || dt < 0 || !std::isfinite(dmax) || !(dmax > 0) ||
      !std::isfinite(ftol) || ftol < 0)
    return IONTRAP_EINVAL;
  if (h->status) return h->status;
  if (!(h->p.flags & (IONTRAP_PSEUDO | IONTRAP_RF_OFF | IONTRAP_TRAP_OFF))) return IONTRAP_EINVAL;
  int st = iontrap_sync(h);
  if (st) return st;
  DeviceGuard g(h->device);
  const size_t vec = 3 * (size_t)h->n * sizeof(double);
  if (!h->d_out && dev_alloc(h, &h->d_out, vec) != cudaSuccess) return IONTRAP_ENOMEM;
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, min_scratch_bytes(h->n)) != cudaSuccess) return IONTRAP_ENOMEM;
  const double step_dt = dt > 0 ? dt : h->p.dt;
  const int b = (int)(h->step & 1);  // the pair stream of parity n holds x_n
  std::vector<unsigned char> hs(min_state_bytes());
  long long done = 0;
  double fn = 0.0;
  int conv = 0;
  cudaError_t e = cudaMemsetAsync(scratch, 0, min_scratch_bytes(h->n), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_v, 0, vec, h->stream);  // from rest
  if (e == cudaSuccess && (h->p.flags & IONTRAP_COULOMB_OFF)) e = cudaMemsetAsync(h->d_out, 0, vec, h->stream);
  if (e == cudaSuccess) e = launch_prep(h, b);
  constexpr int64_t kChunk = 64;
  for (int64_t launched = 0; e == cudaSuccess && launched < max_iters;) {
    // up to kChunk iterations, then a look at the device state
    const int64_t k = std::min<int64_t>(kChunk, max_iters - launched);
    for (int64_t q = 0; q < k && e == cudaSuccess; ++q) {
      if (!(h->p.flags & IONTRAP_COULOMB_OFF)) e = launch_mode(h, MODE_FORCES, h->d_out);
      if (e == cudaSuccess)
        e = launch_min_iteration(h->args, h->d_out, scratch, step_dt, dmax, ftol, h->f64, b, h->stream);
    }
    launched += k;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), scratch, hs.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) break;
    min_progress(hs.data(), &done, &fn, &conv);
    if (conv) break;
  }
  if (e == cudaSuccess && !conv) {
    // |F| at the final positions (the force kernel of one more iteration; it moves
    // nothing when converged, and otherwise the count of moves is already max_iters)
    if (!(h->p.flags & IONTRAP_COULOMB_OFF)) e = launch_mode(h, MODE_FORCES, h->d_out);
    if (e == cudaSuccess)
      e = launch_min_iteration(h->args, h->d_out, scratch, step_dt, dmax, std::numeric_limits<double>::infinity(),
                               h->f64, b, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), scratch, hs.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) {
      long long d2;
      int c2;
      min_progress(hs.data(), &d2, &fn, &c2);
    }
  }
  cudaFree(scratch);
  if (e != cudaSuccess) return cuda_status(h, e);
  if (iters) *iters = done;
  if (fnorm) *fnorm = fn;
  // the minimum at rest: v = 0, a_n evaluated under the handle's forces
  e = cudaMemsetAsync(h->d_v, 0, vec, h->stream);
  if (e != cudaSuccess) return cuda_status(h, e);
  return reevaluate(h);
}

int iontrap_hessian(iontrap_t* h, double* H) {
  if (!h || !H) return IONTRAP_EINVAL;
  if (h->n > 8192) return IONTRAP_ETOOLARGE;
  if (!(h->p.flags & (IONTRAP_PSEUDO | IONTRAP_RF_OFF | IONTRAP_TRAP_OFF))) return IONTRAP_EINVAL;
  int st = iontrap_sync(h);
  if (st) return st;
  DeviceGuard g(h->device);
  const size_t bytes = 9 * (size_t)h->n * (size_t)h->n * sizeof(double);
  double* d_H = nullptr;
  if (cudaMalloc(&d_H, bytes) != cudaSuccess) return IONTRAP_ENOMEM;
  StepArgs a = h->args;
  if (h->p.flags & IONTRAP_COULOMB_OFF)
    for (int s = 0; s < IONTRAP_MAX_SPECIES; ++s) a.spc[s].z = 0.0;
  cudaError_t e = launch_hessian(a, d_H, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(H, d_H, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d_H);
  if (e != cudaSuccess) return cuda_status(h, e);
  return h->status;
}

int iontrap_step_record(iontrap_t* h, int64_t n_steps, int64_t every, uint32_t fields, int64_t avg_steps,
                        double* d_out) {
  if (!h || !d_out || n_steps < 0 || every < 1 || n_steps % every != 0) return IONTRAP_EINVAL;
  const uint32_t known = IONTRAP_REC_X | IONTRAP_REC_V | IONTRAP_REC_VAVG;
  if (fields == 0 || (fields & ~known)) return IONTRAP_EINVAL;
  const bool avg = fields & IONTRAP_REC_VAVG;
  if (avg && (avg_steps < 1 || avg_steps > every)) return IONTRAP_EINVAL;
  if (h->status) return h->status;
  DeviceGuard g(h->device);
  const size_t n3 = 3 * (size_t)h->n;
  if (avg && !h->d_snap && dev_alloc(h, &h->d_snap, 2 * n3 * sizeof(double)) != cudaSuccess) return IONTRAP_ENOMEM;
  const int nf = ((fields & IONTRAP_REC_X) ? 1 : 0) + ((fields & IONTRAP_REC_V) ? 1 : 0) + (avg ? 1 : 0);
  for (int64_t k = 0; k < n_steps / every; ++k) {
    int st;
    if (avg) {
      if (every > avg_steps && (st = iontrap_step(h, every - avg_steps))) return st;
      cudaError_t e = launch_snapshot(h->n, h->d_x, h->d_v, h->d_a, h->d_snap, h->p.dt, h->stream);
      if (e != cudaSuccess) return cuda_status(h, e);
      if ((st = iontrap_step(h, avg_steps))) return st;
    } else if ((st = iontrap_step(h, every))) {
      return st;
    }
    cudaError_t e = launch_record(h->n, h->d_x, h->d_v, h->d_a, h->d_snap, d_out + (size_t)k * nf * n3, fields,
                                  avg ? avg_steps : 0, h->p.dt, h->stream);
    if (e != cudaSuccess) return cuda_status(h, e);
  }
  return h->status;
}

int iontrap_sync(iontrap_t* h) {
  if (!h) return IONTRAP_EINVAL;
  DeviceGuard g(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(h, e);
  int err = 0;
  e = cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(h, e);
  if (err & ERR_TIMEOUT) set_status(h, IONTRAP_ETIMEOUT);
  if (err & ERR_NONFINITE) set_status(h, IONTRAP_ENONFINITE);
  return h->status;
}

int iontrap_state(iontrap_t* h, double* x, double* v, int64_t* step, double* t) {
  if (!h) return IONTRAP_EINVAL;
  const int st = iontrap_sync(h);
  if (st != IONTRAP_OK && st != IONTRAP_ENONFINITE && st != IONTRAP_ETIMEOUT) return st;
  DeviceGuard g(h->device);
  const size_t vec = 3 * (size_t)h->n * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (x) e = cudaMemcpy(x, h->d_x, vec, cudaMemcpyDeviceToHost);
  if (v && e == cudaSuccess) e = cudaMemcpy(v, h->d_v, vec, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(h, e);
  long long dstep = 0;
  e = cudaMemcpy(&dstep, h->d_step, sizeof(dstep), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(h, e);
  if (dstep != h->step && h->status == IONTRAP_OK) set_status(h, IONTRAP_ETIMEOUT);
  if (step) *step = dstep;
  if (t) *t = (double)dstep * h->p.dt;
  return h->status;
}

int iontrap_forces(iontrap_t* h, double* acc) {
  if (!h || !acc) return IONTRAP_EINVAL;
  int st = iontrap_sync(h);
  if (st) return st;
  DeviceGuard g(h->device);
  const size_t vec = 3 * (size_t)h->n * sizeof(double);
  if (!h->d_out && dev_alloc(h, &h->d_out, vec) != cudaSuccess) return IONTRAP_ENOMEM;
  if (h->p.flags & IONTRAP_COULOMB_OFF) {
    std::memset(acc, 0, vec);
    return IONTRAP_OK;
  }
  // the buffer of parity (n & 1) is free at state n
  cudaError_t e = launch_prep(h, (int)(h->step & 1));
  if (e == cudaSuccess) e = launch_mode(h, MODE_FORCES, h->d_out);
  if (e == cudaSuccess) e = cudaMemcpyAsync(acc, h->d_out, vec, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(h, e);
  return iontrap_sync(h);
}

int iontrap_checkpoint(iontrap_t* h, double* x, double* v, double* a, int64_t* step) {
  if (!h) return IONTRAP_EINVAL;
  int st = iontrap_state(h, x, v, step, nullptr);
  if (st) return st;
  DeviceGuard g(h->device);
  if (a) {
    cudaError_t e = cudaMemcpy(a, h->d_a, 3 * (size_t)h->n * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(h, e);
  }
  return h->status;
}

int iontrap_restore(iontrap_t* h, const double* x, const double* v, const double* a, int64_t step) {
  if (!h || !x || !v || !a || step < 0) return IONTRAP_EINVAL;
  for (int64_t k = 0; k < 3 * h->n; ++k)
    if (!std::isfinite(x[k]) || !std::isfinite(v[k]) || !std::isfinite(a[k])) return IONTRAP_EINVAL;
  int st = iontrap_sync(h);
  if (st) return st;
  DeviceGuard g(h->device);
  const size_t vec = 3 * (size_t)h->n * sizeof(double);
  long long s = step;
  cudaError_t e = cudaMemcpyAsync(h->d_x, x, vec, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_v, v, vec, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_a, a, vec, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_step, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = launch_restore(h, (int)((step + 1) & 1));
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(h, e);
  h->step = step;
  return h->status;
}

int iontrap_test_stall(iontrap_t* h, int64_t wait_limit_ns, int32_t cta, int64_t step) {
  if (!h || wait_limit_ns < 0 || step < 0 || (h->fused != 4 && h->fused != 5)) return IONTRAP_EINVAL;
  const int ctas = h->fused == 4 ? h->gp.G : h->rp.G;
  if (cta >= ctas || ctas < 2) return IONTRAP_EINVAL;  // one CTA waits on no other
  if (h->status) return h->status;
  DeviceGuard g(h->device);
  const cudaError_t e = cudaStreamSynchronize(h->stream);  // launches already queued keep their settings
  if (e != cudaSuccess) return cuda_status(h, e);
  h->args.wait_ns = (unsigned long long)wait_limit_ns;
  h->args.stall_on = cta >= 0 ? 1 : 0;
  h->args.stall_cta = cta >= 0 ? cta : 0;
  h->args.stall_step = step;
  return IONTRAP_OK;
}

int iontrap_trace_step(iontrap_t* h, unsigned long long* marks, int64_t cap, int64_t* n_force, int64_t* n_epi) {
  if (!h || !marks || cap < 1 || h->fused == 4) return IONTRAP_EINVAL;
  int st = iontrap_sync(h);
  if (st) return st;
  DeviceGuard g(h->device);
  if (h->fused == 5) {  // one launch of kRpTraceSteps steps, 4 marks per CTA and step
    constexpr int64_t kRpTraceSteps = 8;
    const int64_t nf = 4 * (int64_t)h->rp.G * kRpTraceSteps;
    if (nf > cap) return IONTRAP_EINVAL;
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, nf * sizeof(unsigned long long)) != cudaSuccess) return IONTRAP_ENOMEM;
    cudaError_t e = cudaMemsetAsync(d, 0, nf * sizeof(unsigned long long), h->stream);
    StepArgs a = h->args;
    a.mode = MODE_STEP;
    a.out = nullptr;
    a.trace = d;
    if (e == cudaSuccess)
      e = launch_rp_of(h, a, kRpTraceSteps, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(marks, d, nf * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_status(h, e);
    h->step += kRpTraceSteps;
    if (n_force) *n_force = nf;
    if (n_epi) *n_epi = 0;
    return iontrap_sync(h);
  }
  const dim3 grid = grid_of(h);
  const int64_t nf = 4 * (int64_t)grid.x * grid.y;
  const int64_t ne = h->fused ? 0 : 2 * cdiv(h->n, 32);
  if (nf + ne > cap) return IONTRAP_EINVAL;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, (nf + ne) * sizeof(unsigned long long)) != cudaSuccess) return IONTRAP_ENOMEM;
  cudaError_t e = cudaMemsetAsync(d, 0, (nf + ne) * sizeof(unsigned long long), h->stream);
  StepArgs a = h->args;
  a.mode = MODE_STEP;
  a.out = nullptr;
  a.trace = d;
  a.trace_epi = nf;
  if (e == cudaSuccess) e = launch_step_on(h, a, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(marks, d, (nf + ne) * sizeof(unsigned long long),
                                            cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_status(h, e);
  h->step += 1;
  if (n_force) *n_force = nf;
  if (n_epi) *n_epi = ne;
  return iontrap_sync(h);
}

int iontrap_step_many(iontrap_t* const* hs, const int64_t* n_steps, int count) {
  if (!hs || !n_steps || count < 0) return IONTRAP_EINVAL;
  for (int k = 0; k < count; ++k)
    if (!hs[k] || n_steps[k] < 0) return IONTRAP_EINVAL;
  int first = IONTRAP_OK;
  std::vector<int> batch;
  for (int k = 0; k < count; ++k) {
    iontrap* h = hs[k];
    if (h->status) {
      if (!first) first = h->status;
      continue;
    }
    if (!h->f64 && h->n <= batched_max_n() && n_steps[k] > 0 && h->device == hs[0]->device)
      batch.push_back(k);
    else if (n_steps[k] > 0) {
      const int st = iontrap_step(h, n_steps[k]);
      if (st && !first) first = st;
    }
  }
  if (batch.empty()) return first;
  iontrap* h0 = hs[batch[0]];
  DeviceGuard g(h0->device);
  cudaStream_t st0 = h0->stream;
  std::vector<BatchEns> ens(batch.size());
  std::vector<long long> steps(batch.size());
  cudaError_t e = cudaSuccess;
  for (size_t b = 0; b < batch.size(); ++b) {
    iontrap* h = hs[batch[b]];
    if (h->stream != st0 && e == cudaSuccess) {  // order after work already queued on h's stream
      cudaEvent_t ev;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(ev, h->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st0, ev, 0);
      cudaEventDestroy(ev);
    }
    BatchEns& E = ens[b];
    std::memset(&E, 0, sizeof(E));
    E.x = h->d_x;
    E.v = h->d_v;
    E.a = h->d_a;
    E.sp = h->d_sp;
    for (int q = 0; q < 2; ++q) {
      E.hi[q] = (float4*)h->d_pair[q];
      E.lo[q] = (float4*)h->d_pair[q] + h->n;
    }
    E.step = h->d_step;
    E.err = h->d_err;
    E.n = h->n;
    E.step0 = h->step;
    E.trap = h->args.trap;
    E.nspecies = h->nspecies;
    E.unitw = h->args.unitw;
    std::memcpy(E.spc, h->args.spc, sizeof(E.spc));
    steps[b] = n_steps[batch[b]];
  }
  if (e == cudaSuccess) e = launch_batched(ens, steps, (int)kGpMaxSteps, st0);
  for (size_t b = 0; b < batch.size(); ++b) {
    iontrap* h = hs[batch[b]];
    if (e != cudaSuccess) {
      cuda_status(h, e);
      continue;
    }
    h->step += steps[b];
    if (h->stream != st0) {  // h's later work waits for the batch
      cudaEvent_t ev;
      cudaError_t e2 = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e2 == cudaSuccess) e2 = cudaEventRecord(ev, st0);
      if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(h->stream, ev, 0);
      cudaEventDestroy(ev);
      if (e2 != cudaSuccess) cuda_status(h, e2);
    }
  }
  if (e != cudaSuccess && !first) first = e == cudaErrorMemoryAllocation ? IONTRAP_ENOMEM : IONTRAP_ECUDA;
  return first;
}

void iontrap_destroy(iontrap_t* h) {
  if (!h) return;
  {
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    free_all(h);
  }
  delete h;
}

int iontrap_normals(uint64_t seed, int64_t counter, const int64_t* ids, int64_t m, int precision, double* z) {
  if (m < 0 || (m > 0 && (!ids || !z)) || (precision != IONTRAP_PREC_FP32 && precision != IONTRAP_PREC_FP64))
    return IONTRAP_EINVAL;
  if (m == 0) return IONTRAP_OK;
  long long* d_ids = nullptr;
  double* d_z = nullptr;
  if (cudaMalloc(&d_ids, m * sizeof(long long)) != cudaSuccess) return IONTRAP_ENOMEM;
  if (cudaMalloc(&d_z, 3 * m * sizeof(double)) != cudaSuccess) {
    cudaFree(d_ids);
    return IONTRAP_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(d_ids, ids, m * sizeof(long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_normals(seed, counter, d_ids, m, precision == IONTRAP_PREC_FP64, d_z, 0);
  if (e == cudaSuccess) e = cudaMemcpy(z, d_z, 3 * m * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d_ids);
  cudaFree(d_z);
  return e == cudaSuccess ? IONTRAP_OK : IONTRAP_ECUDA;
}

int iontrap_estimate_bytes(int64_t n, int precision, int64_t* bytes) {
  if (n < 1 || !bytes || (precision != IONTRAP_PREC_FP32 && precision != IONTRAP_PREC_FP64)) return IONTRAP_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IONTRAP_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  const int f64 = precision == IONTRAP_PREC_FP64;
  int T, I, P, J, F;
  default_config(n, f64, sms, &T, &I, &P, &J, &F);
  iontrap_config tc{};
  GpShape gs;
  RpShape rs;
  if (tuned_config(n, f64, dev, &tc) &&
      (step_kernel(f64, tc.threads, tc.ions_per_thread, tc.packed, tc.fused) ||
       (tc.fused == 4 && gp_shape(n, f64, 0, sms, tc.threads, tc.ions_per_thread, tc.packed, tc.jsplit, &gs)) ||
       (tc.fused == 5 && rp_shape(n, f64, 0, sms, tc.threads, tc.ions_per_thread, tc.packed, tc.jsplit, &rs)))) {
    T = tc.threads, I = tc.ions_per_thread, J = tc.jsplit, F = tc.fused;
  }
  const int64_t splits = F == 5 ? cdiv(n, kRpInitJsplit) : cdiv(n, J);
  int64_t part = splits * n * 32;
  if (F == 5 && rp_shape(n, f64, 0, sms, T, I, P, J, &rs))
    part = std::max<int64_t>(part, (int64_t)rp_scratch_bytes(rs.NP, rs.JP));
  const int64_t iblocks = F >= 4 ? cdiv(n, 256) : cdiv(n, (F == 3 ? 32 : (int64_t)T) * I);
  const int64_t vec = 3 * n * (int64_t)sizeof(double);
  const int64_t pair = n * (int64_t)(f64 ? sizeof(double4_32a) : 2 * sizeof(float4));
  *bytes = 3 * vec + n + 2 * pair + part + iblocks * (int64_t)sizeof(unsigned) + 64 +
           (F >= 4 ? (int64_t)kGpSyncBytes : 0);
  return IONTRAP_OK;
}

int iontrap_autotune(iontrap_t* h, double trial_us, iontrap_config* best, double* best_us) {
  if (!h || !(trial_us > 0)) return IONTRAP_EINVAL;
  int st = iontrap_sync(h);
  if (st) return st;
  const int64_t n = h->n;
  std::vector<double> cx(3 * n), cv(3 * n), ca(3 * n);
  int64_t cstep = 0;
  st = iontrap_checkpoint(h, cx.data(), cv.data(), ca.data(), &cstep);
  if (st) return st;
  iontrap_config orig{};
  iontrap_get_config(h, &orig);
  // candidates
  struct Shape {
    int T, I, P;
  };
  std::vector<Shape> shapes;
  if (h->f64) {
    shapes = {{64, 1, 0}, {128, 1, 0}, {128, 2, 0}, {256, 1, 0}};
  } else {
    const Shape small[] = {{32, 1, 0}, {64, 1, 0}, {128, 1, 0}, {64, 2, 1}, {128, 2, 1}};
    const Shape large[] = {{64, 4, 1}, {128, 4, 1}, {256, 4, 1}, {128, 2, 1}};
    if (n < 16384) {
      for (const Shape& sh : small)
        if ((int64_t)sh.T * sh.I <= std::max<int64_t>(64, 2 * n)) shapes.push_back(sh);
    } else {
      for (const Shape& sh : large) shapes.push_back(sh);
    }
  }
  std::vector<iontrap_config> cands;
  for (const Shape& sh : shapes) {
    const int64_t iblocks = cdiv(n, (int64_t)sh.T * sh.I);
    std::vector<int64_t> splits = {1, 2, 3, 4, 6, 8};
    for (int w = 1; w <= 16; w *= 2) {
      const int64_t S = cdiv((int64_t)w * h->sms, iblocks);
      splits.push_back(S);
      const int64_t g = h->sms / gcd64(iblocks, h->sms);  // grid an exact multiple of the SM count
      splits.push_back(cdiv(S, g) * g);
    }
    std::sort(splits.begin(), splits.end());
    splits.erase(std::unique(splits.begin(), splits.end()), splits.end());
    for (int64_t S : splits) {
      if (S < 1 || S > 64 || S > std::max<int64_t>(1, n / (h->f64 ? 8 : 32))) continue;
      int64_t js = cdiv(n, S);
      if (h->f64 && js > kMaxJsplitF64) continue;
      for (int fused = 2; fused >= (h->f64 ? 1 : 0); --fused) {
        if (fused == 2 && (h->f64 || cdiv(n, js) > kMaxClusterSplits || (h->p.flags & IONTRAP_COULOMB_OFF))) continue;
        if (!fused && cdiv(n, js) > kMaxSplitsUnfused) continue;
        iontrap_config c{sh.T, sh.I, sh.P, (int32_t)js, fused, 0, 1};
        if (step_kernel(h->f64, c.threads, c.ions_per_thread, c.packed, c.fused)) cands.push_back(c);
      }
    }
  }
  if (!h->f64 && !(h->p.flags & IONTRAP_COULOMB_OFF)) {  // cluster + warp-split shapes
    const int cw[][2] = {{1, 2}, {1, 4}, {2, 2}, {2, 4}};
    for (const auto& iw : cw)
      for (int64_t S = 2; S <= kMaxClusterSplits3; S *= 2) {
        if (S > std::max<int64_t>(1, n / 128)) continue;
        iontrap_config c{32 * iw[1], iw[0], iw[0] == 2 ? 1 : 0, (int32_t)cdiv(n, S), 3, 0, 1};
        if (step_kernel(0, c.threads, c.ions_per_thread, c.packed, 3)) cands.push_back(c);
      }
  }
  if (!h->f64 && !(h->p.flags & IONTRAP_COULOMB_OFF)) {  // grid-persistent shapes: one or two CTAs per SM
    for (int W : {8, 16})
      for (int per = 1; per <= 2; ++per) {
        const int64_t S = (int64_t)per * h->sms / cdiv(n, 64 * (int64_t)W);
        if (S < 2) continue;
        iontrap_config c{32 * W, 2, 1, (int32_t)cdiv(n, S), 4, 0, 0};
        GpShape gs;
        if (gp_shape(n, 0, h->p.flags, h->sms, c.threads, 2, 1, c.jsplit, &gs)) cands.push_back(c);
      }
    // row-persistent shapes: the ions spread over every SM and the next three counts
    // (fewer CTAs, fewer idle lanes: N = 4096 runs 28 ions per CTA faster than 27), that
    // count rounded up to a power of two (parts aligned with warps), or 32 per CTA
    int64_t r2 = 1;
    while (r2 < cdiv(n, h->sms)) r2 *= 2;
    std::vector<int64_t> rs;
    for (int64_t d = 0; d < 4; ++d) rs.push_back(cdiv(n, h->sms) + d);
    rs.push_back(r2);
    rs.push_back(32);
    if (n <= 170) rs.push_back(n);  // every ion in one CTA
    std::sort(rs.begin(), rs.end());
    rs.erase(std::unique(rs.begin(), rs.end()), rs.end());
    // (one or two ions per thread)
    for (int W : {8, 16})
      for (int I : {1, 2})
        for (int64_t R : rs) {
          iontrap_config c{32 * W, I, 1, (int32_t)R, 5, 0, 0};
          RpShape rs;
          if (rp_shape(n, 0, h->p.flags, h->sms, c.threads, I, 1, R, &rs)) cands.push_back(c);
        }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return IONTRAP_ECUDA;
  // every candidate is timed in two passes and keeps its faster time, so that a clock
  // ramp or a neighbour's burst during one trial does not decide the choice
  std::vector<double> tc_us(cands.size(), 1e300);
  for (int pass = 0; pass < 2 && !h->status; ++pass) {
   for (size_t ci = 0; ci < cands.size(); ++ci) {
    const iontrap_config& c = cands[ci];
    if (iontrap_set_config(h, &c)) continue;
    // calibrate on a few single launches, then time whole graphs for about trial_us
    if (iontrap_step(h, 2) || iontrap_sync(h)) break;
    cudaEventRecord(e0, h->stream);
    iontrap_step(h, 5);
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double graph_us = ms * 1e3 / 5.0 * kGraphSteps;
    const int64_t reps = std::max<int64_t>(1, std::min<int64_t>(50, (int64_t)(trial_us / std::max(1.0, graph_us))));
    iontrap_step(h, kGraphSteps);  // instantiates the graph outside the timed region
    cudaEventRecord(e0, h->stream);
    iontrap_step(h, reps * kGraphSteps);
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    const double us = ms * 1e3 / (double)(reps * kGraphSteps);
    if (h->status) break;
    tc_us[ci] = std::min(tc_us[ci], us);
    if (iontrap_restore(h, cx.data(), cv.data(), ca.data(), cstep)) break;
   }
  }
  double best_t = 1e300;
  iontrap_config bc = orig;
  for (size_t ci = 0; ci < cands.size(); ++ci)
    if (tc_us[ci] < best_t) {
      best_t = tc_us[ci];
      bc = cands[ci];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (h->status) return h->status;
  st = iontrap_set_config(h, &bc);
  if (!st) st = iontrap_restore(h, cx.data(), cv.data(), ca.data(), cstep);
  if (st) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    iontrap_tuning_entry e{};
    e.precision = h->f64;
    e.log2n = log2_floor(n);
    e.threads = bc.threads, e.ions_per_thread = bc.ions_per_thread, e.packed = bc.packed;
    e.splits = (int32_t)cdiv(n, bc.jsplit), e.fused = bc.fused, e.pdl = bc.pdl, e.graph = bc.graph;
    e.us_per_step = (float)best_t;
    g_tune[TuneKey{h->device, h->f64, e.log2n}] = e;
  }
  if (best) *best = bc;
  if (best_us) *best_us = best_t;
  return IONTRAP_OK;
}

int iontrap_autotune_many(iontrap_t* const* hs, int count, double trial_us) {
  if (!hs || count < 1 || !(trial_us > 0)) return IONTRAP_EINVAL;
  for (int k = 0; k < count; ++k)
    if (!hs[k]) return IONTRAP_EINVAL;
  // the handles the batched launch takes, as iontrap_step_many selects them
  std::vector<iontrap_t*> hv;
  for (int k = 0; k < count; ++k) {
    const int st = iontrap_sync(hs[k]);
    if (st) return st;
    if (!hs[k]->f64 && hs[k]->n <= batched_max_n() && hs[k]->device == hs[0]->device) hv.push_back(hs[k]);
  }
  if (hv.empty()) return IONTRAP_OK;
  DeviceGuard g(hv[0]->device);
  const int dev = hv[0]->device;
  struct Ck {
    std::vector<double> x, v, a;
    int64_t step = 0;
  };
  std::vector<Ck> ck(hv.size());
  for (size_t i = 0; i < hv.size(); ++i) {
    const size_t m = 3 * (size_t)hv[i]->n;
    ck[i].x.resize(m), ck[i].v.resize(m), ck[i].a.resize(m);
    const int st = iontrap_checkpoint(hv[i], ck[i].x.data(), ck[i].v.data(), ck[i].a.data(), &ck[i].step);
    if (st) return st;
  }
  auto restore_all = [&]() -> int {
    for (size_t i = 0; i < hv.size(); ++i) {
      const int st = iontrap_restore(hv[i], ck[i].x.data(), ck[i].v.data(), ck[i].a.data(), ck[i].step);
      if (st) return st;
    }
    return IONTRAP_OK;
  };
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return IONTRAP_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return IONTRAP_ECUDA;
  }
  std::vector<int64_t> steps(hv.size());
  // us per step of one batched launch of every handle (the batch runs on the first
  // handle's stream)
  auto time_batch = [&](int64_t nsteps, double* us) -> int {
    std::fill(steps.begin(), steps.end(), nsteps);
    if (cudaEventRecord(e0, hv[0]->stream) != cudaSuccess) return IONTRAP_ECUDA;
    int st = iontrap_step_many(hv.data(), steps.data(), (int)hv.size());
    if (cudaEventRecord(e1, hv[0]->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
      return IONTRAP_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *us = ms * 1e3 / (double)nsteps;
    if (!st) st = restore_all();
    return st;
  };
  auto set_entry = [&](int b, int C, int NP, float us) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    iontrap_tuning_entry e{};
    e.precision = IONTRAP_TUNE_BATCHED;
    e.log2n = b;
    e.threads = 256, e.ions_per_thread = NP, e.packed = 1, e.splits = C, e.fused = 6, e.pdl = 0, e.graph = 0;
    e.us_per_step = us;
    g_tune[TuneKey{dev, IONTRAP_TUNE_BATCHED, b}] = e;
  };
  // buckets of the part-major groups present (256 < n), largest first, with their largest n
  std::map<int, int64_t, std::greater<int>> nmax;
  for (iontrap_t* h : hv)
    if (h->n > 256) {
      const int b = log2_floor(h->n);
      nmax[b] = std::max(nmax[b], h->n);
    }
  int st = IONTRAP_OK;
  double us = 0.0;
  st = time_batch(20, &us);  // warm-up and calibration
  const int64_t nsteps = std::max<int64_t>(20, std::min<int64_t>(1000, (int64_t)(trial_us / std::max(us, 1e-3))));
  for (const auto& bn : nmax) {
    if (st) break;
    const int b = bn.first;
    std::vector<std::pair<int, int>> cands;
    for (int C : {2, 4, 8})
      for (int NP : {0, 2, 4, 6, 8, 12})
        if (batched_shape_fits(bn.second, C, NP) && batched_shape_fits(std::max<int64_t>(257, 1LL << b), C, NP))
          cands.push_back({C, NP});
    std::vector<double> best_us(cands.size(), 1e300);
    for (int pass = 0; pass < 2 && !st; ++pass)
      for (size_t c = 0; c < cands.size() && !st; ++c) {
        set_entry(b, cands[c].first, cands[c].second, 0.f);
        st = time_batch(nsteps, &us);
        best_us[c] = std::min(best_us[c], us);
      }
    if (st) break;
    size_t bc = 0;
    for (size_t c = 1; c < cands.size(); ++c)
      if (best_us[c] < best_us[bc]) bc = c;
    if (!cands.empty()) set_entry(b, cands[bc].first, cands[bc].second, (float)best_us[bc]);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!st) st = restore_all();
  return st;
}

int iontrap_tuning_get(iontrap_tuning_entry* out, int cap, int* count) {
  if (!count || cap < 0 || (cap > 0 && !out)) return IONTRAP_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IONTRAP_ECUDA;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  int k = 0;
  for (const auto& kv : g_tune)
    if (kv.first.dev == dev) {
      if (k < cap) out[k] = kv.second;
      ++k;
    }
  *count = k;
  return IONTRAP_OK;
}

int iontrap_tuning_put(const iontrap_tuning_entry* in, int count) {
  if (count < 0 || (count > 0 && !in)) return IONTRAP_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IONTRAP_ECUDA;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (int k = 0; k < count; ++k) {
    const iontrap_tuning_entry& e = in[k];
    if ((e.precision < 0 || e.precision > IONTRAP_TUNE_BATCHED) || e.log2n < 0 || e.log2n > 40 || e.splits < 0)
      return IONTRAP_EINVAL;
    if (e.splits == 0)
      g_tune.erase(TuneKey{dev, e.precision, e.log2n});
    else
      g_tune[TuneKey{dev, e.precision, e.log2n}] = e;
  }
  return IONTRAP_OK;
}

int iontrap_device_bytes(const iontrap_t* h, int64_t* bytes) {
  if (!h || !bytes) return IONTRAP_EINVAL;
  const int64_t vec = 3 * h->n * (int64_t)sizeof(double);
  const int64_t pair = h->n * (int64_t)(h->f64 ? sizeof(double4_32a) : 2 * sizeof(float4));
  *bytes = 3 * vec + (h->d_out ? vec : 0) + (h->d_snap ? 2 * vec : 0) + h->n + 2 * pair + (int64_t)h->part_bytes +
           (int64_t)h->cnt_len * (int64_t)sizeof(unsigned) + 64 + (h->d_gsync ? (int64_t)kGpSyncBytes : 0);
  return IONTRAP_OK;
}

int iontrap_default_config(int64_t n, int precision, uint32_t flags, int allow_persistent, iontrap_config* c) {
  if (n < 1 || !c || (precision != IONTRAP_PREC_FP32 && precision != IONTRAP_PREC_FP64)) return IONTRAP_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IONTRAP_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  if (prepare_kernels()) return IONTRAP_ECUDA;
  *c = iontrap_config{};
  default_config(n, precision == IONTRAP_PREC_FP64, sms, &c->threads, &c->ions_per_thread, &c->packed, &c->jsplit,
                 &c->fused, (flags & IONTRAP_COULOMB_OFF) ? 0 : allow_persistent);
  if ((flags & IONTRAP_COULOMB_OFF) && c->fused >= 2) c->threads = 64, c->ions_per_thread = 1, c->packed = 0, c->fused = 1;
  c->pdl = 0;
  c->graph = 1;
  return IONTRAP_OK;
}

int iontrap_get_config(const iontrap_t* h, iontrap_config* c) {
  if (!h || !c) return IONTRAP_EINVAL;
  c->threads = h->T;
  c->ions_per_thread = h->I;
  c->packed = h->packed;
  c->jsplit = h->jsplit;
  c->fused = h->fused;
  c->pdl = h->pdl;
  c->graph = h->use_graph;
  return IONTRAP_OK;
}

int iontrap_set_config(iontrap_t* h, const iontrap_config* c) {
  if (!h || !c) return IONTRAP_EINVAL;
  GpShape gs;
  RpShape rs;
  if (c->fused == 4) {
    if (!gp_shape(h->n, h->f64, h->p.flags, h->sms, c->threads, c->ions_per_thread, c->packed, c->jsplit, &gs))
      return IONTRAP_EINVAL;
  } else if (c->fused == 5) {
    if (!rp_shape(h->n, h->f64, h->p.flags, h->sms, c->threads, c->ions_per_thread, c->packed, c->jsplit, &rs))
      return IONTRAP_EINVAL;
  } else if (!step_kernel(h->f64, c->threads, c->ions_per_thread, c->packed, c->fused)) {
    return IONTRAP_EINVAL;
  }
  if (c->jsplit < 1 || c->jsplit > h->n || (h->f64 && c->jsplit > kMaxJsplitF64)) return IONTRAP_EINVAL;
  if (!c->fused && cdiv(h->n, c->jsplit) > kMaxSplitsUnfused) return IONTRAP_EINVAL;
  if (c->fused == 2 && cdiv(h->n, c->jsplit) > kMaxClusterSplits) return IONTRAP_EINVAL;
  if (c->fused == 3 && cdiv(h->n, c->jsplit) > kMaxClusterSplits3) return IONTRAP_EINVAL;
  if ((c->fused >= 2) && (h->p.flags & IONTRAP_COULOMB_OFF)) return IONTRAP_EINVAL;
  if (h->status) return h->status;
  DeviceGuard g(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(h, e);
  h->T = c->threads;
  h->I = c->ions_per_thread;
  h->packed = c->packed;
  h->jsplit = c->jsplit;
  h->fused = c->fused;
  h->pdl = c->pdl ? 1 : 0;
  h->use_graph = c->graph ? 1 : 0;
  destroy_graph(h);
  const int st = alloc_scratch(h);
  if (st) return set_status(h, st);
  return h->status;
}

}  // extern "C"
