/*
 * fp32_pairs.c -- CPU emulation of the FP32 pair arithmetic of the GPU force kernels,
 * for the horizon test in test_fp32_horizon.py.  TEST CODE: it shares nothing with the
 * library (which it never calls) and nothing with the oracle (which it never changes).
 *
 * The Coulomb pair term of Eq. 4, S_i = sum_{j != i} z_j (x_i - x_j) / |x_i - x_j|^3, is
 * evaluated the way an FP32 kernel with hi/lo positions and compensated accumulation
 * does, with every FP32 operation correctly rounded (plain C float arithmetic under
 * -ffp-contract=off, fmaf for the fused multiply-adds):
 *   hi = fl32(x), lo = fl32(x - hi)
 *   d  = (x_j,hi - x_i,hi) + (x_j,lo - x_i,lo)                     per component
 *   r2 = fma(dx, dx, fma(dy, dy, dz dz))
 *   y  = an FP32 approximation of r2^(-1/2)                        (see below)
 *   s  = z_j y (y y),  acc += s d                                   (fma)
 * j runs in ascending order in chunks of 128; within a chunk even and odd j go to two
 * accumulators (as the packed kernels do), whose sum is added to the ion's running sum
 * by Kahan's compensated addition.  The result is returned as FP64 c_i S_i.
 *
 * The reciprocal square root y, by mode:
 *   0  correctly rounded: fl32(1 / sqrt(r2)) evaluated in FP64
 *   1  a hardware-approximation model: the correctly rounded value times
 *      (1 + u 2^-22.9), u uniform in (-1, 1) from a hash of (i, j, salt) -- 2^-22.9 is the
 *      documented maximum relative error of PTX rsqrt.approx.f32
 *   2  mode 1 refined by one Newton-Raphson step folded into the cube (the variant the
 *      library can switch on): e = fma(-r2, y y, 1), s = fma(s0, 1.5 e, s0) with
 *      s0 = z_j y (y y), since (1 - e)^(-3/2) = 1 + 1.5 e + O(e^2)
 */
#include <math.h>
#include <stdint.h>

static inline uint64_t mix64(uint64_t z)
{
    /* SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014) */
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline float rsqrt_model(float r2, int mode, int64_t i, int64_t j, uint64_t salt)
{
    const float cr = (float)(1.0 / sqrt((double)r2));
    if (mode == 0) return cr;
    const uint64_t h = mix64(mix64((uint64_t)i * 0x100000001B3ull ^ salt) ^ (uint64_t)j);
    const double u = ((double)(h >> 11) * 0x1.0p-53) * 2.0 - 1.0; /* (-1, 1) */
    return (float)((double)cr * (1.0 + u * exp2(-22.9)));
}

void emu_coulomb(int64_t n, const double *x, const double *coul, const float *w, int mode,
                 uint64_t salt, double *acc)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        float nh[3], nl[3];
        for (int c = 0; c < 3; ++c) {
            const double xi = x[c * n + i];
            const float h = (float)xi;
            nh[c] = -h;
            nl[c] = -(float)(xi - (double)h);
        }
        float ks[3] = {0.f, 0.f, 0.f}, kc[3] = {0.f, 0.f, 0.f};
        for (int64_t c0 = 0; c0 < n; c0 += 128) {
            const int64_t c1 = c0 + 128 < n ? c0 + 128 : n;
            float ae[3] = {0.f, 0.f, 0.f}, ao[3] = {0.f, 0.f, 0.f};
            for (int64_t j = c0; j < c1; ++j) {
                if (j == i) continue;
                float d[3];
                for (int c = 0; c < 3; ++c) {
                    const double xj = x[c * n + j];
                    const float h = (float)xj;
                    const float l = (float)(xj - (double)h);
                    d[c] = (h + nh[c]) + (l + nl[c]);
                }
                const float r2 = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
                const float y = rsqrt_model(r2, mode == 2 ? 1 : mode, i, j, salt);
                const float y2 = y * y;
                float s = (w[j] * y) * y2;
                if (mode == 2) {
                    const float e = fmaf(-r2, y2, 1.0f);
                    s = fmaf(s, 1.5f * e, s);
                }
                float *a = (j & 1) ? ao : ae;
                for (int c = 0; c < 3; ++c) a[c] = fmaf(s, d[c], a[c]);
            }
            for (int c = 0; c < 3; ++c) {
                const float t = ae[c] + ao[c];
                const float y = t - kc[c];
                const float u = ks[c] + y;
                kc[c] = (u - ks[c]) - y;
                ks[c] = u;
            }
        }
        /* the accumulators hold -S_i (differences taken as x_j - x_i) */
        for (int c = 0; c < 3; ++c) acc[c * n + i] = coul[i] * ((double)kc[c] - (double)ks[c]);
    }
}
