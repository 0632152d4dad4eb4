// libmgq Wilson loops and rethermalisation diagnostics (Sec. III: Wilson
// lines and m x n loops, partial plaquettes W^{1x1}_d, displaced loops
// W^{2x2}_d; Sec. IV.C: smoothness s_p = N_c [1 - W^{1x1}_p] and
// h = max_p s_p).  Measurement kernels: one thread per site, FP64 sums.
#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

// Product of the links along the straight path of `len` steps in direction
// mu starting at x (coordinates updated in place to the end point).
template <class T, int NP>
__device__ __forceinline__ M3<T> line(const Links<T, NP>& U, const Geom& g, int x[4], int mu, int len) {
    M3<T> L = unit3<T>();
    for (int k = 0; k < len; k++) {
        const int lex = lex_of(g, x);
        const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
        L = mul_nn(L, U.load(mu, par, lex >> 1));
#pragma unroll
        for (int d = 0; d < 4; d++)
            if (d == mu) x[d] = wrap(x[d] + 1, g.L[d]);
    }
    return L;
}

// (1/3) Re Tr L^m_mu(x) L^n_nu(x+m mu) [L^n_nu(x) L^m_mu(x+n nu)]^+
template <class T, int NP>
__device__ __forceinline__ double loop_mn(const Links<T, NP>& U, const Geom& g, const int x[4], int mu, int nu, int m, int n) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    const M3<T> a1 = line(U, g, y, mu, m);
    const M3<T> a2 = line(U, g, y, nu, n);
    int z[4] = {x[0], x[1], x[2], x[3]};
    const M3<T> b1 = line(U, g, z, nu, n);
    const M3<T> b2 = line(U, g, z, mu, m);
    return (double)retr_nd(mul_nn(a1, a2), mul_nn(b1, b2)) / 3.0;
}

template <class T, int NP>
__global__ void __launch_bounds__(128) k_wilson_loop(Links<T, NP> U, Geom g, int m, int n, double* __restrict__ partials) {
    double acc = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.V; idx += gridDim.x * blockDim.x) {
        const int par = idx >= g.Vh, h = idx - par * g.Vh;
        int x[4];
        cb_coords(g, par, h, x);
#pragma unroll 1
        for (int mu = 0; mu < 3; mu++)
#pragma unroll 1
            for (int nu = mu + 1; nu < 4; nu++) acc += loop_mn(U, g, x, mu, nu, m, n);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// 8 class sums (W1x1 by chi_munu = 0..2, W2x2 by chi = 0..4) and max s_p:
// partials[q * gridDim.x + block] for q = 0..7, maxima in partials[8 * gridDim.x + block]
template <class T, int NP>
__global__ void __launch_bounds__(128) k_partial_loops(Links<T, NP> U, Geom g, double* __restrict__ partials) {
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double hmax = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.V; idx += gridDim.x * blockDim.x) {
        const int par = idx >= g.Vh, h = idx - par * g.Vh;
        int x[4];
        cb_coords(g, par, h, x);
        const int chi = (x[0] & 1) + (x[1] & 1) + (x[2] & 1) + (x[3] & 1);
#pragma unroll 1
        for (int mu = 0; mu < 3; mu++)
#pragma unroll 1
            for (int nu = mu + 1; nu < 4; nu++) {
                int cmn = 0;
#pragma unroll
                for (int r = 0; r < 4; r++)
                    if (r != mu && r != nu) cmn += x[r] & 1;
                const double w1 = loop_mn(U, g, x, mu, nu, 1, 1);
                const double w2 = loop_mn(U, g, x, mu, nu, 2, 2);
#pragma unroll
                for (int d = 0; d < 3; d++)
                    if (d == cmn) a[d] += w1;
#pragma unroll
                for (int d = 0; d < 5; d++)
                    if (d == chi) a[3 + d] += w2;
                hmax = fmax(hmax, 3.0 * (1.0 - w1));
            }
    }
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const double s = block_sum(a[q]);
        if (threadIdx.x == 0) partials[q * gridDim.x + blockIdx.x] = s;
    }
    __shared__ double smax[128];
    smax[threadIdx.x] = hmax;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[8 * gridDim.x + blockIdx.x] = smax[0];
}

__global__ void k_max_final(const double* __restrict__ partials, int n, double* out) {
    __shared__ double sm[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, partials[i]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sm[0];
}

static double binom(int n, int k) {
    double r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

}  // namespace mgq

using namespace mgq;

extern "C" {

mgq_status mgq_wilson_loop(const mgq_lattice* lat, int m, int n, double* out, void* stream) {
    Trace trace("mgq_wilson_loop");
    mgq_status s = check_lattice(lat, true, "mgq_wilson_loop");
    if (s) return s;
    if (m < 1 || n < 1 || m > 64 || n > 64) return fail(MGQ_EINVAL, "mgq_wilson_loop: need 1 <= m, n <= 64");
    if (!out) return fail(MGQ_EINVAL, "mgq_wilson_loop: out is NULL");
    const Geom g = make_geom(lat->dims);
    cudaStream_t st = as_stream(stream);
    const int nb = reduction_blocks(g.V, 128);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_wilson_loop<T, NP><<<nb, 128, 0, st>>>(links_of<T, NP>(lat), g, m, n, ws_partials(lat));
    });
    double* sc = ws_scalars(lat);
    launch_final_sum(ws_partials(lat), nb, 1.0 / (6.0 * (double)g.V), sc + 24, st);
    if ((s = cuda_check("mgq_wilson_loop"))) return s;
    return deliver(sc + 24, out, 1, st, "mgq_wilson_loop");
}

mgq_status mgq_partial_loops(const mgq_lattice* lat, double* out, void* stream) {
    Trace trace("mgq_partial_loops");
    mgq_status s = check_lattice(lat, true, "mgq_partial_loops");
    if (s) return s;
    if (!out) return fail(MGQ_EINVAL, "mgq_partial_loops: out is NULL");
    const Geom g = make_geom(lat->dims);
    cudaStream_t st = as_stream(stream);
    int nb = reduction_blocks(g.V, 128);
    if (nb > (int)(WS_NPARTIALS / 9)) nb = (int)(WS_NPARTIALS / 9);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_partial_loops<T, NP><<<nb, 128, 0, st>>>(links_of<T, NP>(lat), g, ws_partials(lat));
    });
    double* sc = ws_scalars(lat);
    const double V = (double)g.V;
    for (int d = 0; d < 3; d++)
        launch_final_sum(ws_partials(lat) + d * nb, nb, 1.0 / (2.0 * (4 - d) * (3 - d) * binom(4, d) * V / 16.0),
                         sc + 24 + d, st);
    for (int d = 0; d < 5; d++)
        launch_final_sum(ws_partials(lat) + (3 + d) * nb, nb, 1.0 / (6.0 * binom(4, d) * V / 16.0), sc + 27 + d, st);
    k_max_final<<<1, 256, 0, st>>>(ws_partials(lat) + 8 * nb, nb, sc + 32);
    if ((s = cuda_check("mgq_partial_loops"))) return s;
    return deliver(sc + 24, out, 9, st, "mgq_partial_loops");
}

}  // extern "C"
