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

// =============================================================== heat bath
// One link: V = U A; per subgroup (0,1), (0,2), (1,2): w from the block,
// k = 2 beta |w| / 3, up to n_hb Creutz attempts
//   a0 = 1 + log1p((1 - u0) expm1(-2k)) / k, accept iff u1^2 <= 1 - a0^2,
// direction cos(theta) = 2 u2 - 1, phi = 2 pi u3; R = X (w/|w|), U <- R U,
// V <- R V; reunitarise at the end.  dec[s] = accepted attempt or 255.
template <class T>
__device__ __forceinline__ void hb_link(M3<T>& u, const M3<T>& A, T beta, int n_hb, const RngKey& rk, uint32_t lex,
                                        uint32_t mu, uint8_t* dec) {
    M3<T> v = mul_nn(u, A);
#pragma unroll
    for (int s = 0; s < 3; s++) {
        const int i = (s == 2) ? 1 : 0, j = (s == 0) ? 1 : 2;
        T w[4];
        block_w(v, i, j, w);
        const T xi = m_sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        uint8_t d = 255;
        if (xi >= tiny_norm<T>()) {
            const T k = T(2) * beta * xi / T(3);
            const T em = m_expm1(T(-2) * k);
            for (int att = 0; att < n_hb; att++) {
                const uint4 r = draw(rk, lex, mu, (uint32_t)s, (uint32_t)att, KIND_HB);
                const T u0 = u01<T>(r.x), u1 = u01<T>(r.y), u2 = u01<T>(r.z), u3 = u01<T>(r.w);
                const T a0 = T(1) + m_log1p((T(1) - u0) * em) / k;
                const T rest = sub_rn(T(1), mul_rn(a0, a0));
                if (mul_rn(u1, u1) <= rest) {
                    const T rad = m_sqrt(rest);
                    const T ct = T(2) * u2 - T(1);
                    const T st = m_sqrt(sub_rn(T(1), mul_rn(ct, ct)));
                    T sp, cp;
                    m_sincospi(T(2) * u3, &sp, &cp);
                    const T X[4] = {a0, rad * st * cp, rad * st * sp, rad * ct};
                    const T inv = T(1) / xi;
                    const T wh[4] = {w[0] * inv, w[1] * inv, w[2] * inv, w[3] * inv};
                    T R[4];
                    qmul(X, wh, R);
                    left_su2(u, i, j, R);
                    left_su2(v, i, j, R);
                    d = (uint8_t)att;
                    break;
                }
            }
        }
        if (dec) dec[s] = d;
    }
    reunitarize(u);
}

// Overrelaxation of one link: per subgroup R = (w/|w|)^2; reunitarise.
template <class T>
__device__ __forceinline__ void or_link(M3<T>& u, const M3<T>& A) {
    M3<T> v = mul_nn(u, A);
#pragma unroll
    for (int s = 0; s < 3; s++) {
        const int i = (s == 2) ? 1 : 0, j = (s == 0) ? 1 : 2;
        T w[4];
        block_w(v, i, j, w);
        const T n2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
        if (!(m_sqrt(n2) >= tiny_norm<T>())) continue;
        const T inv2 = T(1) / n2;
        // (w/|w|)^2 = (w0^2 - |w_vec|^2, 2 w0 w_vec) / |w|^2
        const T R[4] = {(w[0] * w[0] - w[1] * w[1] - w[2] * w[2] - w[3] * w[3]) * inv2, T(2) * w[0] * w[1] * inv2,
                        T(2) * w[0] * w[2] * inv2, T(2) * w[0] * w[3] * inv2};
        left_su2(u, i, j, R);
        left_su2(v, i, j, R);
    }
    reunitarize(u);
}

}  // namespace mgq
