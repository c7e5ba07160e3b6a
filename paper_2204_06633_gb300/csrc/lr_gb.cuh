// Galactic-binary polarisations generated on the device (Sec. "Template generation"): the
// source-frame waveform A cos Phi, A sin Phi with Phi(t) = 2 pi (f0 t + fdot t^2/2 + fddot t^3/6)
// + phi0, weighted by (1 + cos^2 iota) and 2 cos iota.  These are the un-rotated polarisations the
// response takes as input (psi rotates the antenna patterns inside the response).
//
// Accuracy: the phase in cycles, f0 t ~ 3e5 at one year and 10 mHz, would carry ~3e-11 cycles of
// FP64 rounding (a white ~2e-10 relative error of h that the TDI cancellation amplifies), so it is
// formed in double-double: t = t0 + i dt from the exact product i * dt (two_prod by FMA) and an
// exact two_sum, f0 t and fdot t^2 / 2 as double-double products, the tiny fddot term in FP64.
// The cycle count is then reduced modulo one exactly (the integer nearest the high word is
// subtracted without rounding) and 2 pi frac + phi0 goes to the FP64 sincos: the phase error is a
// few 1e-16 rad for any t and f.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lisaresp.h"

namespace lr {

struct GbConst {
    double ap, ax;     // A (1 + cos^2 iota), 2 A cos iota
    double f0, fd2;    // f0, fdot / 2
    double fdd6;       // fddot / 6
    double phi0;
};

__host__ __device__ inline GbConst make_gb(const lr_gb &g)
{
    const double ci = cos(g.iota);
    return {g.A * (1.0 + ci * ci), 2.0 * g.A * ci, g.f0, 0.5 * g.fdot, g.fddot / 6.0, g.phi0};
}

// h+, hx at t = t0 + i dt
__device__ __forceinline__ void gb_strain(const GbConst &g, double t0, double dt, int64_t i, double &hp,
                                          double &hc)
{
    // t = th + tl exactly (i dt as a double-double product, then an exact two_sum with t0)
    const double fi = (double)i;
    const double p = fi * dt, pe = fma(fi, dt, -p);
    const double th = t0 + p, bb = th - t0;
    const double tl = ((t0 - (th - bb)) + (p - bb)) + pe;
    // f0 t: double-double product; fdot t^2 / 2: t^2 as a double-double, times fdot / 2
    const double c1 = g.f0 * th, c1e = fma(g.f0, th, -c1);
    const double t2 = th * th, t2e = fma(th, th, -t2) + 2.0 * th * tl;
    const double c2 = g.fd2 * t2, c2e = fma(g.fd2, t2, -c2) + g.fd2 * t2e;
    const double s = c1 + c2, sb = s - c1;
    const double se = (c1 - (s - sb)) + (c2 - sb);
    const double lo = se + (c1e + g.f0 * tl) + c2e + g.fdd6 * t2 * th;
    // modulo one cycle: s - rint(s) is exact
    const double frac = (s - rint(s)) + lo;
    double sn, cs;
    sincos(fma(6.283185307179586, frac, g.phi0), &sn, &cs);
    hp = g.ap * cs;
    hc = g.ax * sn;
}

}  // namespace lr
