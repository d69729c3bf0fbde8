// claw_interp.cuh -- the coarse-to-fine space-time interpolation of a fine ghost cell (Sec. 2.2:
// ghosts not covered by the level come from the coarser level, interpolated in space and time),
// shared by the ghost-fill kernel, its adjoint and the pulled-ghost step, so that all three take
// the same value and the same minmod branches.
//   time:  Q(tau) = (1 - tau) Q_c^n + tau Q_c^{n+1} at the coarse parent and its four neighbours
//   space: q_f = Q + xi sx + eta sy, sx = minmod(Q_e - Q, Q - Q_w), sy likewise (conservative,
//          exact for linear data); xi, eta the fine centre's offset in coarse cells
// A coarse neighbour across a solid wall carries its normal velocity negated (sflags), as does a
// fine ghost across one (flags).
#pragma once

#include "claw_internal.h"

namespace claw {

__device__ __forceinline__ double interp_minmod(double a, double b)
{
    if (!(a * b > 0.0)) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

// -1 for the velocity component m (1: u, 2: v) that a wall flips (flags bit0: u, bit1: v)
__device__ __forceinline__ double interp_sign(int flags, int m)
{
    return ((m == 1 && (flags & 1)) || (m == 2 && (flags & 2))) ? -1.0 : 1.0;
}

// the five coarse values of component m at time fraction tau: centre, west, east, south, north
__device__ __forceinline__ void interp_coarse(const InterpCell& C, int m, const double* cold, const double* cnew,
                                              double tau, double Q[5])
{
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const long long o = C.src[s] + m * C.splane[s];
        Q[s] = interp_sign(C.sflags[s], m) * fma(tau, cnew[o], (1.0 - tau) * cold[o]);
    }
}

// component m of the fine ghost value
__device__ __forceinline__ double interp_value(const InterpCell& C, int m, const double* cold, const double* cnew,
                                               double tau)
{
    double Q[5];
    interp_coarse(C, m, cold, cnew, tau, Q);
    const double sx = interp_minmod(Q[2] - Q[0], Q[0] - Q[1]);
    const double sy = interp_minmod(Q[4] - Q[0], Q[0] - Q[3]);
    return interp_sign(C.flags, m) * fma(C.eta, sy, fma(C.xi, sx, Q[0]));
}

}  // namespace claw
