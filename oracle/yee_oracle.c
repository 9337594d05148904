/*
 * Plain CPU oracle of the 3-D Yee FDTD leapfrog sweep (Sec. 2.1 of Cessenat,
 * "Sophie, an FDTD code on the way to multicore"), in double (_f64) and
 * single (_f32) precision. Each update uses one fused multiply-add (C's
 * fma / fmaf, correctly rounded by definition), every other operation is
 * rounded separately.
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code, header or table
 * with the CUDA path. Build with -ffp-contract=off so that no other a*b+c is
 * fused: only the explicit fma/fmaf calls are.
 *
 * Pins (checked by tests/ with -m "not gpu"):
 *   - exact discrete cavity eigenmodes (closed form) in vacuum and in a uniform
 *     dielectric, and the scalar recurrence of a lossy mode (a1, a2, Ca, Cb);
 *   - the discrete energy balance with loss and a source (a2, a4, a7);
 *   - conservation of the node divergence of eps*E (a1-a3);
 *   - adjointness of the two discrete curls (a1 vs a2 index conventions);
 *   - the 4-cell edge average against a 2x2 box filter (material reading);
 *   - the waveform against its closed form.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define C0 299792458.0
#define EPS0 8.8541878128e-12

#define REAL double
#define SUF f64
#define FMA fma
#include "yee_oracle_body.h"
#undef REAL
#undef SUF
#undef FMA

#define REAL float
#define SUF f32
#define FMA fmaf
#include "yee_oracle_body.h"
#undef REAL
#undef SUF
#undef FMA

/*
 * Source waveform values s[m] = amp * w((n0 + m + 1/2) * dt), m in [0, n).
 * kind 0 (Gaussian-modulated sine): w(t) = sin(2 pi f0 (t-t0)) exp(-(t-t0)^2 / (2 st^2))
 * kind 1 (Gaussian pulse):          w(t) = exp(-(t-t0)^2 / (2 st^2))
 * with st = 1/(2 pi sf), sf = bw / (2 sqrt(2 ln 2)): bw is the full width at
 * half maximum of the amplitude spectrum of the envelope.
 */
void oracle_waveform(int kind, double amp, double f0, double bw, double t0, double dt,
                     long n0, long n, double *out)
{
    const double pi = 3.14159265358979323846;
    const double sf = bw / (2.0 * sqrt(2.0 * log(2.0)));
    const double st = 1.0 / (2.0 * pi * sf);
    for (long m = 0; m < n; ++m) {
        const double t = ((double)(n0 + m) + 0.5) * dt;
        const double u = t - t0;
        const double env = exp(-(u * u) / (2.0 * st * st));
        out[m] = amp * (kind == 0 ? sin(2.0 * pi * f0 * u) * env : env);
    }
}

/*
 * The 24-bit storage form of the precision study (not in the paper; the
 * north-star's reduced-storage form): every stored field value keeps the upper
 * 24 bits of its float (sign, exponent, 15 mantissa bits). A value v is first
 * rounded to 16 significant bits by Veltkamp's splitting (Dekker, "A
 * floating-point technique for extending the available precision", 1971):
 * with sigma = 2^8 + 1, c = sigma * v, hi = c + (v - c), three float
 * operations each rounded to nearest (this file is compiled without
 * contraction), which leaves hi with at most 24 - 8 = 16 significant bits;
 * the low 8 bits of hi's pattern, zero for normal values, are then dropped
 * (for subnormal values the split is not exact and the drop truncates).
 * Rounds a[0..n) in place.
 */
void oracle_round24_f32(float *a, long n)
{
    for (long i = 0; i < n; ++i) {
        const float v = a[i];
        const float c = 257.0f * v;
        const float d = v - c;
        const float hi = c + d;
        uint32_t u;
        memcpy(&u, &hi, 4);
        u &= 0xFFFFFF00u;
        memcpy(&a[i], &u, 4);
    }
}

int oracle_abi_version(void) { return 1; }
