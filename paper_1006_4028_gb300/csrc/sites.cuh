// Even-odd site indexing shared by the stencil kernels: the coordinates of
// an output half-site and the half-site indices of its 8 neighbours (layout
// in dp_internal.h: half-site s = lexicographic index >> 1 per parity).
#pragma once

#include "dp_internal.h"

namespace dp {

// site coordinates and the half-site indices of its 8 neighbours
// (half-site indices fit in 32 bits: V/2 < 2^31 for every allowed geometry)
struct Nbr {
    int t, x, y, z;
    int f[4], b[4];  // forward / backward neighbour per direction
};

__device__ __forceinline__ Nbr neighbours(const Geom &g, long long s64, int parity)
{
    Nbr o;
    const unsigned s = (unsigned)s64;
    const int xh = (int)(s % (unsigned)g.Lxh);
    unsigned q = s / (unsigned)g.Lxh;
    o.y = (int)(q % (unsigned)g.Ly);
    q /= (unsigned)g.Ly;
    o.z = (int)(q % (unsigned)g.Lz);
    o.t = (int)(q / (unsigned)g.Lz);
    o.x = 2 * xh + ((o.t + o.y + o.z + parity) & 1);
    auto row = [&](int tt, int zz, int yy) -> int {
        return ((tt * g.Lz + zz) * g.Ly + yy) * g.Lxh;
    };
    const int tp = (o.t + 1 == g.T) ? 0 : o.t + 1, tm = (o.t == 0) ? g.T - 1 : o.t - 1;
    const int xp = (o.x + 1 == g.Lx) ? 0 : o.x + 1, xm = (o.x == 0) ? g.Lx - 1 : o.x - 1;
    const int yp = (o.y + 1 == g.Ly) ? 0 : o.y + 1, ym = (o.y == 0) ? g.Ly - 1 : o.y - 1;
    const int zp = (o.z + 1 == g.Lz) ? 0 : o.z + 1, zm = (o.z == 0) ? g.Lz - 1 : o.z - 1;
    const int r0 = row(o.t, o.z, o.y);
    o.f[0] = row(tp, o.z, o.y) + xh;
    o.b[0] = row(tm, o.z, o.y) + xh;
    o.f[1] = r0 + (xp >> 1);
    o.b[1] = r0 + (xm >> 1);
    o.f[2] = row(o.t, o.z, yp) + xh;
    o.b[2] = row(o.t, o.z, ym) + xh;
    o.f[3] = row(o.t, zp, o.y) + xh;
    o.b[3] = row(o.t, zm, o.y) + xh;
    return o;
}

}  // namespace dp
