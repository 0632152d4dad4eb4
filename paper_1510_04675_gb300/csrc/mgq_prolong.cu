// libmgq multiscale maps (Sec. III): restriction (Eq. restriction), the
// transfer step of the prolongation (Eq. prolongation) and the interpolation
// stages, each a repeated Jacobi APE step (Eq. APE) on the active bonds of
// stage d that minimises the partial action S_d (Eq. smoothing).
#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

// P_SU(3)(M): Gram-Schmidt start W, then NPASS passes over the subgroups
// (0,1), (0,2), (1,2) of W <- R W with R = R(w/|w|) maximising Re Tr(R W M^+).
template <class T>
__device__ __forceinline__ M3<T> su3_project(const M3<T>& M) {
    constexpr int NPASS = 8;
    M3<T> W = M;
    reunitarize(W);
#pragma unroll 1
    for (int pass = 0; pass < NPASS; pass++) {
#pragma unroll
        for (int s = 0; s < 3; s++) {
            const int i = (s == 2) ? 1 : 0, j = (s == 0) ? 1 : 2;
            const M3<T> V = mul_nd(W, M);
            T w[4];
            block_w(V, i, j, w);
            const T xi = m_sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
            if (!(xi >= tiny_norm<T>())) continue;
            const T inv = T(1) / xi;
            const T r[4] = {w[0] * inv, w[1] * inv, w[2] * inv, w[3] * inv};
            left_su2(W, i, j, r);
        }
    }
    return W;
}

// number of odd coordinates of x other than those in directions a and b
__device__ __forceinline__ int odd_count_except(const int x[4], int a, int b) {
    int c = 0;
#pragma unroll
    for (int r = 0; r < 4; r++)
        if (r != a && r != b) c += x[r] & 1;
    return c;
}

// Transfer: U^f_mu(n) = U^c_mu(n/2) where every coordinate of n is even,
// U^f_mu(n + e_mu) = 1 there, and every other fine bond = 1.
template <class T, int NP>
__global__ void k_transfer(Links<T, NP> Uc, Geom gc, Links<T, NP> Uf, Geom gf) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * gf.Vh) return;
    const int mp = idx / gf.Vh, h = idx - mp * gf.Vh, mu = mp >> 1, par = mp & 1;
    int x[4];
    cb_coords(gf, par, h, x);
    M3<T> u = unit3<T>();
    if (((x[0] | x[1] | x[2] | x[3]) & 1) == 0) {
        const int xc[4] = {x[0] >> 1, x[1] >> 1, x[2] >> 1, x[3] >> 1};
        const int lc = lex_of(gc, xc);
        u = Uc.load(mu, (xc[0] + xc[1] + xc[2] + xc[3]) & 1, lc >> 1);
    }
    Uf.store(mu, par, h, u);
}

// Restriction: U^c_mu(n/2) = U^f_mu(n) U^f_mu(n + e_mu) at n with all coordinates even.
template <class T, int NP>
__global__ void k_restrict(Links<T, NP> Uf, Geom gf, Links<T, NP> Uc, Geom gc) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * gc.Vh) return;
    const int mp = idx / gc.Vh, h = idx - mp * gc.Vh, mu = mp >> 1, par = mp & 1;
    int xc[4];
    cb_coords(gc, par, h, xc);
    const int xf[4] = {2 * xc[0], 2 * xc[1], 2 * xc[2], 2 * xc[3]};
    const int lf = lex_of(gf, xf);
    const int lf1 = lex_hop(gf, xf, mu, +1);
    M3<T> u = mul_nn(Uf.load(mu, 0, lf >> 1), Uf.load(mu, 1, lf1 >> 1));
    if (sizeof(T) == 4) reunitarize(u);
    Uc.store(mu, par, h, u);
}

// One Jacobi APE step of stage d: for every bond with chi_mu(n) = d + 1,
// Unew = P_SU(3)[U + c sum_{nu != mu, n_nu odd} (T+_munu + T-_munu)],
// T+ = U_nu(n) U_mu(n+nu) U_nu(n+mu)^+, T- = U_nu(n-nu)^+ U_mu(n-nu) U_nu(n-nu+mu);
// reads Uin, writes only the active bonds of Uout.
template <class T, int NP>
__global__ void __launch_bounds__(128) k_ape(Links<T, NP> Uin, Links<T, NP> Uout, Geom g, int d, T c) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * g.Vh) return;
    const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
    int x[4];
    cb_coords(g, par, h, x);
    if (odd_count_except(x, mu, mu) != d + 1) return;
    const int op = par ^ 1;
    M3<T> M = Uin.load(mu, par, h);
    const int lpm = lex_hop(g, x, mu, +1);
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu || !(x[nu] & 1)) continue;
        const int lpn = lex_hop(g, x, nu, +1), lmn = lex_hop(g, x, nu, -1);
        const int lmn_pm = lex_hop(g, x, nu, -1, mu, +1);
        const M3<T> tp = mul_nd(mul_nn(Uin.load(nu, par, h), Uin.load(mu, op, lpn >> 1)), Uin.load(nu, op, lpm >> 1));
        const M3<T> tm = mul_nn(mul_dn(Uin.load(nu, op, lmn >> 1), Uin.load(mu, op, lmn >> 1)),
                                Uin.load(nu, par, lmn_pm >> 1));
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const Cx<T> sum = tp.e[i][j] + tm.e[i][j];
                M.e[i][j] = M.e[i][j] + scale(sum, c);
            }
    }
    Uout.store(mu, par, h, su3_project(M));
}

// Partial action S_d / beta = sum over plaquettes with chi_munu(n) = d of (1 - Re Tr U_p / 3).
template <class T, int NP>
__global__ void __launch_bounds__(256) k_partial_action(Links<T, NP> U, Geom g, int d, double* __restrict__ partials) {
    double acc = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.V; idx += gridDim.x * blockDim.x) {
        const int par = idx >= g.Vh, h = idx - par * g.Vh;
        int x[4];
        cb_coords(g, par, h, x);
        const int op = par ^ 1;
#pragma unroll
        for (int mu = 0; mu < 3; mu++) {
#pragma unroll
            for (int nu = mu + 1; nu < 4; nu++) {
                if (odd_count_except(x, mu, nu) != d) continue;
                const int hpm = lex_hop(g, x, mu, +1) >> 1, hpn = lex_hop(g, x, nu, +1) >> 1;
                const M3<T> a = mul_nn(U.load(mu, par, h), U.load(nu, op, hpm));
                const M3<T> b = mul_nn(U.load(nu, par, h), U.load(mu, op, hpn));
                acc += 1.0 - (double)retr_nd(a, b) / 3.0;
            }
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

static mgq_status partial_action_into(const mgq_lattice* lat, const void* links, int d, double* partials, double* out,
                                      cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    const int nb = reduction_blocks(g.V, 256);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_partial_action<T, NP><<<nb, 256, 0, st>>>(links_at<T, NP>(const_cast<void*>(links), lat->dims), g, d, partials);
    });
    launch_final_sum(partials, nb, 1.0, out, st);
    return cuda_check("partial_action");
}

}  // namespace mgq

using namespace mgq;

extern "C" {

mgq_status mgq_restrict(const mgq_lattice* fine, mgq_lattice* coarse, void* stream) {
    Trace trace("mgq_restrict");
    mgq_status s = check_lattice(fine, false, "mgq_restrict");
    if (s) return s;
    if ((s = check_lattice(coarse, false, "mgq_restrict"))) return s;
    for (int mu = 0; mu < 4; mu++)
        if (fine->dims[mu] != 2 * coarse->dims[mu])
            return fail(MGQ_EINVAL, "mgq_restrict: fine extents must be twice the coarse extents");
    if (fine->prec != coarse->prec) return fail(MGQ_EINVAL, "mgq_restrict: precisions differ");
    const Geom gf = make_geom(fine->dims), gc = make_geom(coarse->dims);
    cudaStream_t st = as_stream(stream);
    dispatch_prec(fine->prec, [&]<class T, int NP>() {
        k_restrict<T, NP><<<nblk(8L * gc.Vh, 128), 128, 0, st>>>(links_of<T, NP>(fine), gf, links_of<T, NP>(coarse), gc);
    });
    return cuda_check("mgq_restrict");
}

mgq_status mgq_prolongate(const mgq_lattice* coarse, mgq_lattice* fine, double c, double rel_tol, int max_iter,
                          int* iters_out, double* sd_out, void* stream) {
    Trace trace("mgq_prolongate");
    mgq_status s = check_lattice(coarse, false, "mgq_prolongate");
    if (s) return s;
    if ((s = check_lattice(fine, true, "mgq_prolongate"))) return s;
    for (int mu = 0; mu < 4; mu++)
        if (fine->dims[mu] != 2 * coarse->dims[mu])
            return fail(MGQ_EINVAL, "mgq_prolongate: fine extents must be twice the coarse extents");
    if (fine->prec != coarse->prec) return fail(MGQ_EINVAL, "mgq_prolongate: precisions differ");
    if (!(c > 0.0) || max_iter < 0) return fail(MGQ_EINVAL, "mgq_prolongate: need c > 0 and max_iter >= 0");
    const Geom gf = make_geom(fine->dims), gc = make_geom(coarse->dims);
    cudaStream_t st = as_stream(stream);
    const uint64_t lb = links_bytes(fine);
    void* bufs[2] = {fine->links, ws_links(fine)};
    double* sc = ws_scalars(fine);
    double host_sd[2];
    dispatch_prec(fine->prec, [&]<class T, int NP>() {
        k_transfer<T, NP><<<nblk(8L * gf.Vh, 128), 128, 0, st>>>(links_of<T, NP>(coarse), gc, links_of<T, NP>(fine), gf);
    });
    if ((s = cuda_check("mgq_prolongate: transfer"))) return s;
    int cur = 0;
    for (int d = 0; d <= 2; d++) {
        // both buffers hold the full field: inactive bonds never change during the stage
        if (cudaMemcpyAsync(bufs[1 - cur], bufs[cur], lb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return cuda_check("mgq_prolongate: copy");
        if ((s = partial_action_into(fine, bufs[cur], d, ws_partials(fine), sc + 20, st))) return s;
        double prev = 0.0, now = 0.0;
        if (rel_tol > 0.0) {
            if ((s = deliver(sc + 20, &prev, 1, st, "mgq_prolongate"))) return s;
        }
        int it = 0;
        while (it < max_iter) {
            dispatch_prec(fine->prec, [&]<class T, int NP>() {
                k_ape<T, NP><<<nblk(8L * gf.Vh, 128), 128, 0, st>>>(links_at<T, NP>(bufs[cur], fine->dims),
                                                                    links_at<T, NP>(bufs[1 - cur], fine->dims), gf, d, (T)c);
            });
            if ((s = cuda_check("mgq_prolongate: ape"))) return s;
            cur = 1 - cur;
            it++;
            if (rel_tol > 0.0) {
                if ((s = partial_action_into(fine, bufs[cur], d, ws_partials(fine), sc + 20, st))) return s;
                if ((s = deliver(sc + 20, &now, 1, st, "mgq_prolongate"))) return s;
                const bool done = fabs(now - prev) <= rel_tol * fabs(prev);
                prev = now;
                if (done) break;
            }
        }
        if (iters_out) iters_out[d] = it;
        if (sd_out) {
            if ((s = partial_action_into(fine, bufs[cur], d, ws_partials(fine), sc + 20, st))) return s;
            if ((s = deliver(sc + 20, host_sd, 1, st, "mgq_prolongate"))) return s;
            sd_out[d] = host_sd[0];
        }
    }
    if (cur != 0) {
        if (cudaMemcpyAsync(fine->links, bufs[cur], lb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return cuda_check("mgq_prolongate: copy back");
    }
    return MGQ_OK;
}

}  // extern "C"
