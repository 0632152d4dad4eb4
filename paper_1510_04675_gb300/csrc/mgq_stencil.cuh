// Stencils shared by the libmgq kernels: the staple sum (Sec. III, Wilson
// action), the per-site plaquette sum, and the clover field strength.
#pragma once

#include "mgq_device.cuh"

namespace mgq {

// =============================================================== staple
// A_mu(x) = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
//                          + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) ]
// so that Re Tr(U_mu(x) A_mu(x)) sums the six plaquettes holding U_mu(x).
// x has parity par; x +- e_nu has parity 1 - par, x + e_mu - e_nu parity par.
template <class T, int NP>
__device__ __forceinline__ M3<T> staple(const Links<T, NP>& U, const Geom& g, const int x[4], int h, int mu, int par) {
    M3<T> A;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) A.e[i][j] = mk(T(0), T(0));
    const int op = par ^ 1;
    const int hpm = lex_hop(g, x, mu, +1) >> 1;
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        const int hpn = lex_hop(g, x, nu, +1) >> 1;
        const int hmn = lex_hop(g, x, nu, -1) >> 1;
        const int hpm_mn = lex_hop(g, x, mu, +1, nu, -1) >> 1;
        M3<T> up, dn;
        {
            const M3<T> a = U.load(nu, op, hpm);   // U_nu(x+mu)
            const M3<T> b = U.load(mu, op, hpn);   // U_mu(x+nu)
            const M3<T> c = U.load(nu, par, h);    // U_nu(x)
            up = mul_nd(mul_nd(a, b), c);
        }
        {
            const M3<T> d = U.load(nu, par, hpm_mn);  // U_nu(x+mu-nu)
            const M3<T> e = U.load(mu, op, hmn);      // U_mu(x-nu)
            const M3<T> f = U.load(nu, op, hmn);      // U_nu(x-nu)
            dn = mul_nn(mul_dd(d, e), f);
        }
        acc_add(up, dn);
        acc_add(A, up);
    }
    return A;
}

// =============================================================== plaquette
// Per site: sum over mu < nu of Re Tr[U_mu(x) U_nu(x+mu) (U_nu(x) U_mu(x+nu))^+].
template <class T, int NP>
__device__ __forceinline__ double site_plaquettes(const Links<T, NP>& U, const Geom& g, int par, int h) {
    int x[4];
    cb_coords(g, par, h, x);
    const int op = par ^ 1;
    double acc = 0.0;
#pragma unroll
    for (int mu = 0; mu < 3; mu++) {
        const M3<T> umu = U.load(mu, par, h);
        const int hpm = lex_hop(g, x, mu, +1) >> 1;
#pragma unroll
        for (int nu = mu + 1; nu < 4; nu++) {
            const int hpn = lex_hop(g, x, nu, +1) >> 1;
            const M3<T> a = mul_nn(umu, U.load(nu, op, hpm));
            const M3<T> b = mul_nn(U.load(nu, par, h), U.load(mu, op, hpn));
            acc += (double)retr_nd(a, b);
        }
    }
    return acc;
}

}  // namespace mgq
