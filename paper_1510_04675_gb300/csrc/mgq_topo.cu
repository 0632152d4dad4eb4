// libmgq three-loop improved topological charge (Sec. IV.C; the gluonic
// operator of de Forcrand, Garcia Perez and Stamatescu, Nucl. Phys. B 499
// (1997) 409).  q_m(x) is the clover charge density built from the four m x m
// leaves around x in every plane (m = 1, 2, 3).  An m x m clover on spacing a
// is the 1 x 1 clover on spacing m a, so q_m / m^4 = a^4 [q + (m a)^2 X +
// (m a)^4 Y + ...] for a smooth field, and sum_m c_m q_m / m^4 with
// sum c_m = 1, sum c_m m^2 = 0, sum c_m m^4 = 0, i.e. c = (3/2, -3/5, 1/10),
// has no O(a^2) and O(a^4) terms at tree level.
#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

// Product of the links along the m x m leaf l around x in the (mu, nu) plane,
// counterclockwise from x.  The sides follow the cycle +mu, +nu, -mu, -nu
// starting at entry l (l = 0: +mu +nu -mu -nu, l = 1: +nu -mu -nu +mu, ...),
// m links each.  Only the two in-plane coordinates move; a step along +d
// multiplies by U_d(y), a step along -d by U_d(y - d)^+.
template <class T, int NP>
__device__ M3<T> leaf_product(const Links<T, NP>& U, const Geom& g, const int x[4], int mu, int nu, int l, int m) {
    const int st[4] = {1, g.L[0], g.L[0] * g.L[1], g.L[0] * g.L[1] * g.L[2]};
    const int smu = pick(st, mu), snu = pick(st, nu), Lmu = pick(g.L, mu), Lnu = pick(g.L, nu);
    int ya = pick(x, mu), yb = pick(x, nu);
    const int base = lex_of(g, x) - ya * smu - yb * snu;
    const int rest = x[0] + x[1] + x[2] + x[3] - ya - yb;
    M3<T> P = unit3<T>();
#pragma unroll 1
    for (int side = 0; side < 4; side++) {
        const int c = (l + side) & 3;
        const bool along_nu = c & 1;
        const bool fwd = c < 2;
        const int dir = along_nu ? nu : mu;
#pragma unroll 1
        for (int k = 0; k < m; k++) {
            if (!fwd) {
                if (along_nu) yb = yb == 0 ? Lnu - 1 : yb - 1;
                else ya = ya == 0 ? Lmu - 1 : ya - 1;
            }
            const int lex = base + ya * smu + yb * snu;
            const M3<T> u = U.load(dir, (rest + ya + yb) & 1, lex >> 1);
            P = fwd ? mul_nn(P, u) : mul_nd(P, u);
            if (fwd) {
                if (along_nu) yb = yb == Lnu - 1 ? 0 : yb + 1;
                else ya = ya == Lmu - 1 ? 0 : ya + 1;
            }
        }
    }
    return P;
}

// Algebra coefficients of G = traceless part of (Q - Q^+)/8, Q the sum of the
// four m x m leaves (= clover_coeffs for m = 1).
template <class T, int NP>
__device__ void clover_coeffs_m(const Links<T, NP>& U, const Geom& g, const int x[4], int mu, int nu, int m,
                                T out[8]) {
    M3<T> Q = leaf_product(U, g, x, mu, nu, 0, m);
#pragma unroll 1
    for (int l = 1; l < 4; l++) acc_add(Q, leaf_product(U, g, x, mu, nu, l, m));
    ta_coeffs(Q, out);
#pragma unroll
    for (int a = 0; a < 8; a++) out[a] *= T(0.25);
}

// Per site q_m = 1/(8 pi^2) (g01.g23 - g02.g13 + g03.g12) from the m x m
// clover (Tr(X_a X_b) = -delta_ab / 2), m = 1, 2, 3; per-block FP64 partials
// of the three charges at partials[(m - 1) gridDim.x + block].
template <class T, int NP>
__global__ void __launch_bounds__(128) k_topo_improved(Links<T, NP> U, Geom g, double* __restrict__ partials) {
    double q[3] = {0.0, 0.0, 0.0};
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.V; idx += gridDim.x * blockDim.x) {
        const int par = idx >= g.Vh, h = idx - par * g.Vh;
        int x[4];
        cb_coords(g, par, h, x);
#pragma unroll
        for (int m = 1; m <= 3; m++) {
            T d = T(0);
#pragma unroll 1
            for (int p = 0; p < 3; p++) {
                // (01, 23), (02, 13), (03, 12) with signs +, -, +
                const int b0 = p == 0 ? 2 : 1, b1 = p == 2 ? 2 : 3;
                T Ga[8], Gb[8];
                clover_coeffs_m(U, g, x, 0, p + 1, m, Ga);
                clover_coeffs_m(U, g, x, b0, b1, m, Gb);
                T dot = T(0);
#pragma unroll
                for (int a = 0; a < 8; a++) dot += Ga[a] * Gb[a];
                d += p == 1 ? -dot : dot;
            }
            q[m - 1] += (double)d * (1.0 / (8.0 * 9.869604401089358));
        }
    }
#pragma unroll
    for (int m = 0; m < 3; m++) {
        const double v = block_sum(q[m]);
        if (threadIdx.x == 0) partials[m * gridDim.x + blockIdx.x] = v;
    }
}

// out[0] = 3/2 Q_1 - 3/5 Q_2 / 16 + 1/10 Q_3 / 81 from out[1..3]
__global__ void k_improved_combine(double* out) {
    out[0] = 1.5 * out[1] - 0.6 * out[2] / 16.0 + 0.1 * out[3] / 81.0;
}

// {Q_improved, Q_1x1, Q_2x2, Q_3x3} into dev_out[0..3] (device)
mgq_status improved_charge_into(const mgq_lattice* lat, double* partials, double* dev_out, cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    const int nb = reduction_blocks(g.V, 128) < 2048 ? reduction_blocks(g.V, 128) : 2048;
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        k_topo_improved<T, NP><<<nb, 128, 0, st>>>(links_of<T, NP>(lat), g, partials);
    });
    for (int m = 0; m < 3; m++) launch_final_sum(partials + m * nb, nb, 1.0, dev_out + 1 + m, st);
    k_improved_combine<<<1, 1, 0, st>>>(dev_out);
    return cuda_check("improved_charge");
}

}  // namespace mgq

using namespace mgq;

extern "C" {

mgq_status mgq_topo_charge_improved(const mgq_lattice* lat, double* Q_out, void* stream) {
    Trace trace("mgq_topo_charge_improved");
    mgq_status s = check_lattice(lat, true, "mgq_topo_charge_improved");
    if (s) return s;
    if (!Q_out) return fail(MGQ_EINVAL, "mgq_topo_charge_improved: Q_out is NULL");
    cudaStream_t st = as_stream(stream);
    double* sc = ws_scalars(lat);
    if ((s = improved_charge_into(lat, ws_partials(lat), sc + 20, st))) return s;
    return deliver(sc + 20, Q_out, 4, st, "mgq_topo_charge_improved");
}

}  // extern "C"
