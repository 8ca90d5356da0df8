// ew_bc_dev.cuh -- the boundary closure of a box as an extension of the grid
// function beyond its active points, for every kernel that reads or stages
// points outside the box.
//
// Each axis has a lower and an upper face, each of one of two kinds:
//   Dirichlet  the wall point holds u = 0 and is not active; beyond it the
//              odd reflection u(w + d) = -u(w - d) (for the fourth-order
//              stencil this is u = 0 and u_xx = 0 on the wall);
//   Neumann    the wall point is active; beyond it the even reflection
//              u(w + d) = u(w - d): the wall is a symmetry plane (the centred
//              first difference across it vanishes, the condition the paper
//              uses for the symmetry plane of its double-ellipsoid geometry).
// In active-index coordinates 0 .. n-1 the lower wall sits at -1 (Dirichlet)
// or 0 (Neumann), the upper wall at n (Dirichlet) or n-1 (Neumann).  The
// reflections about both walls make the extension periodic with period
// P = 2 (w_hi - w_lo); over one period the sign flips when exactly one face
// is a Dirichlet face.  Every point the stencils can reach, however short the
// axis, maps to an active point with a sign, or to a Dirichlet wall (0).
#pragma once

#include <stdint.h>

namespace ew {

// 2-bit code of axis a in a grid's face mask (bit 2a: lower face Neumann,
// bit 2a+1: upper face Neumann)
__host__ __device__ __forceinline__ int axis_bc(int bc, int a) { return (bc >> (2 * a)) & 3; }

// the active index holding the value of point p of an axis of n active points
// with face code `code`, and its sign; -1 for a Dirichlet wall (value 0)
template <typename I>
__host__ __device__ __forceinline__ I ext_axis(I p, I n, int code, int& sign) {
    const I wl = (code & 1) ? I(0) : I(-1);
    const I wu = (code & 2) ? n - 1 : n;
    const I M = wu - wl, P = 2 * M;
    const I d = p - wl;
    const I k = d >= 0 ? d / P : -((P - 1 - d) / P);  // floor(d / P)
    I t = d - k * P;                                 // 0 <= t < P
    int s = ((k & 1) && (code == 1 || code == 2)) ? -1 : 1;
    if (t > M) {  // beyond the upper wall: reflect about it
        t = P - t;
        if (!(code & 2)) s = -s;
    }
    const I q = wl + t;
    if (q == I(-1) || q == n) return I(-1);
    sign = s;
    return q;
}

}  // namespace ew
