// zm_stencil.cuh -- per-node bodies of the surface-mesh stencil passes (FP64), shared by the
// single-interface kernels (zm_stencil.cu) and the batched kernels (zm_batch.cu):
//   ghost fill two nodes deep (paper Sec. 3.1 BoundaryCondition), 4th-order differences
//   (Sec. 3.1 SurfaceMesh), tangents / metric / normal / sheet strength (Sec. 2 ZModel), the
//   vorticity derivative dw/dt = -2 A grad Phi + mu Lap w and the SSP-RK3 stage combine
//   (Sec. 3.1 TimeIntegrator).
#pragma once

#include "zm_internal.cuh"

namespace zm {

// The five values f[c-2 .. c+2] along one axis of node (i, j), with two-deep ghosts:
// periodic: wrap and add +-seam (the period jump of the field across the seam: L1 for z1 along
// alpha1, L2 for z2 along alpha2, zero otherwise); free edges: odd reflection about the edge
// node, i.e. linear extrapolation f(edge - m) = 2 f(edge) - f(edge + m).
__device__ __forceinline__ void line5(const double *__restrict__ f, int i, int j, int axis,
                                      const Geom &g, double seam, double v[5])
{
    const int n = axis ? g.n2 : g.n1;
    const int c0 = axis ? j : i;
    const size_t stride = axis ? 1 : (size_t)g.n2;
    const double *base = axis ? f + (size_t)i * g.n2 : f + j;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int c = c0 + k - 2;
        if (c >= 0 && c < n) {
            v[k] = base[c * stride];
        } else if (g.periodic) {
            const int cw = (c < 0) ? c + n : c - n;
            v[k] = !ZM_IDX_OK(cw, n) ? 0.0 : (c < 0) ? base[cw * stride] - seam : base[cw * stride] + seam;
        } else {
            const int e = (c < 0) ? 0 : n - 1, m = (c < 0) ? -c : 2 * (n - 1) - c;
            v[k] = ZM_IDX_OK(m, n) ? 2.0 * base[e * stride] - base[m * stride] : 0.0;
        }
    }
}

// 4th-order first and second differences of five samples spaced dx apart.
__device__ __forceinline__ double diff1(const double v[5], double inv12dx)
{
    return ((v[0] - v[4]) + 8.0 * (v[3] - v[1])) * inv12dx;
}
__device__ __forceinline__ double diff2(const double v[5], double inv12dx2)
{
    return (16.0 * (v[1] + v[3]) - (v[0] + v[4]) - 30.0 * v[2]) * inv12dx2;
}

// Geometry of node p: writes q = g z3 + 1/8 w^T h^-1 w and, by kKind,
//   kGeoFp64: FP64 source record (position, scaled strength);
//   kGeoFp32c: FP32 near and far source records, the tile sphere (centre by the tile's middle
//     node, radius by atomicMax) and max |gamma'| (atomicMax, for the fixed-point scale);
//   kGeoLow: unit normal.
constexpr int kGeoFp64 = 0, kGeoFp32c = 1, kGeoLow = 2;

template <int kKind>
__device__ __forceinline__ void geometry_point(const Geom &g, const Tiling &t, int p,
                                               const double *__restrict__ y, double pref,
                                               double grav, float d2f, void *__restrict__ src,
                                               float *__restrict__ far_rec, float4 *__restrict__ tinfo,
                                               unsigned int *gmax, double *__restrict__ q,
                                               double *__restrict__ nrm)
{
    if (!ZM_IDX_OK(p, g.N)) return;
    const int i = p / g.n2, j = p - (p / g.n2) * g.n2;
    const double *z = y, *w = y + 3 * (size_t)g.N;
    const double i12a = g.i12a, i12b = g.i12b;

    double a1[3], a2[3], v[5];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        line5(z + (size_t)c * g.N, i, j, 0, g, c == 0 ? g.L1 : 0.0, v);
        a1[c] = diff1(v, i12a);
        line5(z + (size_t)c * g.N, i, j, 1, g, c == 1 ? g.L2 : 0.0, v);
        a2[c] = diff1(v, i12b);
    }
    const double h11 = a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2];
    const double h12 = a1[0] * a2[0] + a1[1] * a2[1] + a1[2] * a2[2];
    const double h22 = a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2];
    const double det = h11 * h22 - h12 * h12;
    const double w1 = w[p], w2 = w[(size_t)g.N + p];
    const double z3 = z[2 * (size_t)g.N + p];
    const double quad = h22 * w1 * w1 - 2.0 * h12 * w1 * w2 + h11 * w2 * w2;

    if (kKind == kGeoLow) {
        // unit normal; |a1 x a2|^2 = det (Lagrange's identity) also gives 1/det
        const double nx = a1[1] * a2[2] - a1[2] * a2[1];
        const double ny = a1[2] * a2[0] - a1[0] * a2[2];
        const double nz = a1[0] * a2[1] - a1[1] * a2[0];
        const double il = dev::rsqrt_nr(nx * nx + ny * ny + nz * nz);
        q[p] = grav * z3 + 0.125 * quad * (il * il);
        nrm[p] = nx * il;
        nrm[(size_t)g.N + p] = ny * il;
        nrm[2 * (size_t)g.N + p] = nz * il;
        return;
    }
    q[p] = grav * z3 + 0.125 * quad / det;
    // scaled sheet strength gamma' = (dx1 dx2 / 4 pi) (w1 a2 - w2 a1)
    double gm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) gm[c] = pref * (w1 * a2[c] - w2 * a1[c]);

    const int ti = i / t.tp1, tj = j / t.tp2;
    const size_t tile = (size_t)ti * t.nt2 + tj;
    const int slot = (i - ti * t.tp1) * t.tp2 + (j - tj * t.tp2);
    if (!ZM_IDX_OK(tile, t.ntiles) || !ZM_IDX_OK(slot, t.ts)) return;
    if (kKind == kGeoFp32c) {
        // near record: hi/lo position and strength
        float *r = static_cast<float *>(src) + tile * kRec32 * t.ts + slot;
        float gf[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double zc = z[(size_t)c * g.N + p];
            const float hi = __double2float_rn(zc);
            gf[c] = __double2float_rn(gm[c]);
            r[(size_t)c * t.ts] = hi;
            r[(size_t)(3 + c) * t.ts] = __double2float_rn(zc - (double)hi);
            r[(size_t)(6 + c) * t.ts] = gf[c];
        }
        // far record: position relative to the tile centre (the middle node of the tile's part
        // of the mesh), |s|^2 + delta^2, strength and s x strength
        const int h1 = min(t.tp1, g.n1 - ti * t.tp1), h2 = min(t.tp2, g.n2 - tj * t.tp2);
        const size_t pc = (size_t)(ti * t.tp1 + h1 / 2) * g.n2 + (tj * t.tp2 + h2 / 2);
        if (!ZM_IDX_OK(pc, g.N)) return;
        float cf[3], sf[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cf[c] = __double2float_rn(z[(size_t)c * g.N + pc]);
            sf[c] = __double2float_rn(z[(size_t)c * g.N + p] - (double)cf[c]);
        }
        float *f = far_rec + tile * kRec32F * t.ts + slot;
        f[0] = sf[0];
        f[t.ts] = sf[1];
        f[2 * (size_t)t.ts] = sf[2];
        f[3 * (size_t)t.ts] = fmaf(sf[0], sf[0], fmaf(sf[1], sf[1], fmaf(sf[2], sf[2], d2f)));
        // FP32 strength and s x strength
#pragma unroll
        for (int c = 0; c < 3; ++c) f[(size_t)(kFarRowG + c) * t.ts] = gf[c];
        f[(size_t)(kFarRowG + 3) * t.ts] = __double2float_rn((double)sf[1] * gf[2] - (double)sf[2] * gf[1]);
        f[(size_t)(kFarRowG + 4) * t.ts] = __double2float_rn((double)sf[2] * gf[0] - (double)sf[0] * gf[2]);
        f[(size_t)(kFarRowG + 5) * t.ts] = __double2float_rn((double)sf[0] * gf[1] - (double)sf[1] * gf[0]);
        const float rad = sqrtf(sf[0] * sf[0] + sf[1] * sf[1] + sf[2] * sf[2]);
        atomicMax(reinterpret_cast<unsigned int *>(&tinfo[tile].w), __float_as_uint(rad));
        const float gn = sqrtf(gf[0] * gf[0] + gf[1] * gf[1] + gf[2] * gf[2]);
        atomicMax(gmax, __float_as_uint(gn));
        if ((size_t)p == pc) {
            tinfo[tile].x = cf[0];
            tinfo[tile].y = cf[1];
            tinfo[tile].z = cf[2];
        }
    } else {
        double *r = static_cast<double *>(src) + tile * kRec64 * t.ts + slot;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            r[(size_t)c * t.ts] = z[(size_t)c * g.N + p];
            r[(size_t)(3 + c) * t.ts] = gm[c];
        }
    }
}


// Vorticity pass at node p.  mode 0: wdot = dw/dt.  mode 1: yout = ca y0 + cb (y + dt (u, dw/dt)).
template <bool kVisc, int kMode>
__device__ __forceinline__ void vorticity_point(const Geom &g, int p, const double *__restrict__ phi,
                                                const double *__restrict__ y,
                                                const double *__restrict__ u, double atwood,
                                                double mu, double dt, double ca, double cb,
                                                const double *y0, double *yout,
                                                double *__restrict__ wdot)
{
    if (!ZM_IDX_OK(p, g.N)) return;
    const int i = p / g.n2, j = p - (p / g.n2) * g.n2;
    const size_t N = g.N;
    double v[5];
    line5(phi, i, j, 0, g, 0.0, v);
    double f1 = -2.0 * atwood * diff1(v, g.i12a);
    line5(phi, i, j, 1, g, 0.0, v);
    double f2 = -2.0 * atwood * diff1(v, g.i12b);
    if (kVisc) {
        const double ia = g.i12a2, ib = g.i12b2;
        const double *w = y + 3 * N;
        line5(w, i, j, 0, g, 0.0, v);
        double l1 = diff2(v, ia);
        line5(w, i, j, 1, g, 0.0, v);
        l1 += diff2(v, ib);
        line5(w + N, i, j, 0, g, 0.0, v);
        double l2 = diff2(v, ia);
        line5(w + N, i, j, 1, g, 0.0, v);
        l2 += diff2(v, ib);
        f1 += mu * l1;
        f2 += mu * l2;
    }
    if (kMode == 0) {
        wdot[p] = f1;
        wdot[N + p] = f2;
        return;
    }
    const double d[5] = {u[p], u[N + p], u[2 * N + p], f1, f2};
    double out[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c] = ca * y0[c * N + p] + cb * (y[c * N + p] + dt * d[c]);
#pragma unroll
    for (int c = 0; c < 5; ++c) yout[c * N + p] = out[c];
}

}  // namespace zm
