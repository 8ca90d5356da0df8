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
// P = 2 (w_hi - w_lo) (the sign flips once per period when exactly one face is
// a Dirichlet face).  Every point the stencils can reach, however short the
// axis, maps to an active point with a sign, or to a Dirichlet wall (0).
#pragma once

#include <stdint.h>

namespace ew {

// 2-bit code of axis a in a grid's face mask (bit 2a: lower face Neumann,
// bit 2a+1: upper face Neumann)
__host__ __device__ __forceinline__ int axis_bc(int bc, int a) { return (bc >> (2 * a)) & 3; }

// the active index holding the value of point p of an axis of n active points
// with face code `code`, and its sign; -1 for a Dirichlet wall (value 0).
// Two Dirichlet faces take the periodic form in one remainder; an axis with a
// Neumann face reflects about the walls until the point is inside: one
// reflection for any point within an axis length of the box, and every two
// reflections shorten the distance by 2 (w_hi - w_lo), so tiny axes take a few
// more.  (The staging loops of the blocked kernels run this for their halo
// points; its cost shows in their time.)
template <typename I>
__host__ __device__ __forceinline__ I ext_axis(I p, I n, int code, int& sign) {
    if (code == 0) {  // two Dirichlet faces: the odd extension, period 2 (n + 1), in one remainder
        const I P = 2 * (n + 1);
        I q = (p + 1) % P;
        if (q < 0) q += P;
        q -= 1;  // -1 .. 2n
        if (q == I(-1) || q == n) return I(-1);
        if (q < n) {
            sign = 1;
            return q;
        }
        sign = -1;
        return 2 * n - q;
    }
    const I wl = (code & 1) ? I(0) : I(-1);
    const I wu = (code & 2) ? n - 1 : n;
    if (wu <= wl) return I(-1);  // no such axis (grids have w_hi - w_lo >= 2); keeps the loop finite
    int s = 1;
    // bounded: a point 128 axis lengths out needs at most 256 reflections
    for (int it = 0; it < 256 && (p < wl || p > wu); ++it) {
        if (p < wl) {
            p = 2 * wl - p;
            if (!(code & 1)) s = -s;
        } else {
            p = 2 * wu - p;
            if (!(code & 2)) s = -s;
        }
    }
    if (p < wl || p > wu || p == I(-1) || p == n) return I(-1);
    sign = s;
    return p;
}

}  // namespace ew
