// zm_stencil.cu -- surface-mesh stencil kernels (FP64):
//   geometry pass: two-deep ghosts, tangents a1 = D1 z, a2 = D2 z, metric, unit normal, the
//     sheet strength gamma = w1 a2 - w2 a1 written as Birkhoff-Rott source records, and
//     q = g z3 + 1/8 w^T h^-1 w (paper Sec. 2 ZModel "surface normals"; Sec. 3.1 SurfaceMesh
//     two-node-deep stencils and BoundaryCondition ghost rules);
//   reduction of split Birkhoff-Rott partials into u and Phi = q + 1/2 |u|^2;
//   vorticity pass: dw_l/dt = -2 A D_l Phi + mu Lap w_l, fused with the SSP-RK3 stage combine
//     (Sec. 3.1 TimeIntegrator, three derivative evaluations per step).
// One thread per mesh node; neighbours come through L1/L2, so each kernel streams its fields
// once from HBM.
#include "zm_stencil.cuh"

namespace zm {
namespace {

constexpr int kTpb = 256;

template <int kKind>
__global__ void __launch_bounds__(kTpb)
    geometry_kernel(Geom g, Tiling t, const double *__restrict__ y, double pref, double grav,
                    void *__restrict__ src, double *__restrict__ q, double *__restrict__ nrm)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.N) return;
    geometry_point<kKind>(g, t, p, y, pref, grav, 0.0f, src, nullptr, nullptr, nullptr, q, nrm);
}

__global__ void __launch_bounds__(kTpb)
    reduce_kernel(int N, int nsplit, const double *__restrict__ part, const double *__restrict__ q,
                  double *__restrict__ u, double *__restrict__ phi, int write_phi)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < nsplit; ++k) {
#pragma unroll
        for (int c = 0; c < 3; ++c) s[c] += part[((size_t)k * 3 + c) * N + p];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) u[(size_t)c * N + p] = s[c];
    if (write_phi) phi[p] = q[p] + 0.5 * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
}

// The same reduction for many splits and few points (small meshes, where the all-pairs pass
// splits the sources into dozens of slices to fill the GPU): kG threads per point each sum the
// splits g, g + kG, ..., and the kG partial sums are added in a fixed order through shared
// memory, so the result is deterministic (though associated differently from reduce_kernel).
constexpr int kRedG = 8;
__global__ void __launch_bounds__(kTpb)
    reduce_wide_kernel(int N, int nsplit, const double *__restrict__ part, const double *__restrict__ q,
                       double *__restrict__ u, double *__restrict__ phi, int write_phi)
{
    __shared__ double sh[3][kRedG][kTpb / kRedG];
    const int lp = threadIdx.x % (kTpb / kRedG), g = threadIdx.x / (kTpb / kRedG);
    const int p = blockIdx.x * (kTpb / kRedG) + lp;
    double s[3] = {0.0, 0.0, 0.0};
    if (p < N)
        for (int k = g; k < nsplit; k += kRedG) {
#pragma unroll
            for (int c = 0; c < 3; ++c) s[c] += part[((size_t)k * 3 + c) * N + p];
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) sh[c][g][lp] = s[c];
    __syncthreads();
    if (g != 0 || p >= N) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double t = sh[c][0][lp];
        for (int h = 1; h < kRedG; ++h) t += sh[c][h][lp];
        s[c] = t;
        u[(size_t)c * N + p] = t;
    }
    if (write_phi) phi[p] = q[p] + 0.5 * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
}

template <bool kVisc, int kMode>
__global__ void __launch_bounds__(kTpb)
    vorticity_kernel(Geom g, const double *__restrict__ phi, const double *__restrict__ y,
                     const double *__restrict__ u, double atwood, double mu, double dt, double ca,
                     double cb, const double *y0, double *yout, double *__restrict__ wdot)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.N) return;
    vorticity_point<kVisc, kMode>(g, p, phi, y, u, atwood, mu, dt, ca, cb, y0, yout, wdot);
}

__global__ void finite_kernel(size_t n, const double *__restrict__ y, int *bad)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(y[k])) {
            atomicOr(bad, 1);
            return;
        }
}

}  // namespace

int check_finite(zm_ctx *c, const double *y, size_t n, int *dev_flag)
{
    int rc = cuda_check(cudaMemsetAsync(dev_flag, 0, sizeof(int), c->stream), "finite flag clear");
    if (rc) return rc;
    finite_kernel<<<4 * 152, kTpb, 0, c->stream>>>(n, y, dev_flag);
    return cuda_check(cudaGetLastError(), "finite check launch");
}

int launch_geometry(zm_ctx *c, const double *y)
{
    // every buffer a launch below writes must exist (a wiring error returns, never faults)
    if (!y || !c->q || (c->order != ZM_ORDER_HIGH && !c->nrm) ||
        (c->order != ZM_ORDER_LOW && !c->batch && !c->src))
        return set_error(ZM_ERR_INVALID, "geometry pass: missing buffer");
    const Geom &g = c->geom;
    const double pref = g.dx1 * g.dx2 / (4.0 * 3.14159265358979323846);
    dim3 grid((g.N + kTpb - 1) / kTpb);
    cudaEvent_t ev = nullptr;
    prof_begin(c, ZM_K_GEOMETRY, &ev);
    if (c->order != ZM_ORDER_HIGH)
        geometry_kernel<kGeoLow><<<grid, kTpb, 0, c->stream>>>(g, c->tiling, y, pref, c->g, nullptr,
                                                             c->q, c->nrm);
    // FP64 source records (high and medium order); FP32C contexts build theirs in the batch
    if (c->order != ZM_ORDER_LOW && !c->batch) {
        if (c->order == ZM_ORDER_MEDIUM) {  // the second geometry pass of a medium-order evaluation
            prof_end(c, ZM_K_GEOMETRY, ev);
            prof_begin(c, ZM_K_GEOMETRY, &ev);
        }
        geometry_kernel<kGeoFp64><<<grid, kTpb, 0, c->stream>>>(g, c->tiling, y, pref, c->g, c->src,
                                                              c->q, nullptr);
    }
    prof_end(c, ZM_K_GEOMETRY, ev);
    return cuda_check(cudaGetLastError(), "geometry kernel launch");
}

int launch_reduce(zm_ctx *c, bool write_phi)
{
    if (!c->part || !c->u || !c->phi || !c->q) return set_error(ZM_ERR_INVALID, "reduction: missing buffer");
    const Geom &g = c->geom;
    dim3 grid((g.N + kTpb - 1) / kTpb);
    cudaEvent_t ev = nullptr;
    prof_begin(c, ZM_K_REDUCE, &ev);
    if (c->plan.nsplit >= 4 * kRedG && g.N <= 16 * kTpb * 152)
        reduce_wide_kernel<<<(g.N + kTpb / kRedG - 1) / (kTpb / kRedG), kTpb, 0, c->stream>>>(
            g.N, c->plan.nsplit, c->part, c->q, c->u, c->phi, write_phi ? 1 : 0);
    else
        reduce_kernel<<<grid, kTpb, 0, c->stream>>>(g.N, c->plan.nsplit, c->part, c->q, c->u, c->phi,
                                                    write_phi ? 1 : 0);
    prof_end(c, ZM_K_REDUCE, ev);
    return cuda_check(cudaGetLastError(), "reduce kernel launch");
}

int launch_vorticity(zm_ctx *c, const double *y, double *wdot_out, const double *y0, double *yout,
                     double dt, double ca, double cb, int mode)
{
    if (!y || !c->phi || !c->u || (mode == 0 && !wdot_out) || (mode == 1 && (!y0 || !yout)))
        return set_error(ZM_ERR_INVALID, "vorticity pass: missing buffer");
    const Geom &g = c->geom;
    dim3 grid((g.N + kTpb - 1) / kTpb);
    cudaEvent_t ev = nullptr;
    prof_begin(c, ZM_K_VORT, &ev);
    const bool visc = (c->mu != 0.0);
#define ZM_VORT(V, M)                                                                          \
    vorticity_kernel<V, M><<<grid, kTpb, 0, c->stream>>>(g, c->phi, y, c->u, c->atwood, c->mu, \
                                                         dt, ca, cb, y0, yout, wdot_out)
    if (mode == 0) {
        if (visc) ZM_VORT(true, 0); else ZM_VORT(false, 0);
    } else {
        if (visc) ZM_VORT(true, 1); else ZM_VORT(false, 1);
    }
#undef ZM_VORT
    prof_end(c, ZM_K_VORT, ev);
    return cuda_check(cudaGetLastError(), "vorticity kernel launch");
}

ZM_BOUNDS_READER(bounds_stencil)

}  // namespace zm
