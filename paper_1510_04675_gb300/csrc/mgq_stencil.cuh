// Stencils shared by the libmgq kernels: the staple sum (Sec. III, Wilson
// action), the per-site plaquette sum, and the clover field strength.
#pragma once

#include "mgq_device.cuh"

namespace mgq {

// Rows 0 and 1 of a b^+ and of a b (row 2 of the result is left unset): the
// callers rebuild it as conj(row0 x row1) because the product is in SU(3).
template <class T> __device__ __forceinline__ M3<T> mul_nd_2(const M3<T>& a, const M3<T>& b) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            r.e[i][j] = mulc(a.e[i][0], b.e[j][0]) + mulc(a.e[i][1], b.e[j][1]) + mulc(a.e[i][2], b.e[j][2]);
    return r;
}
template <class T> __device__ __forceinline__ M3<T> mul_nn_2(const M3<T>& a, const M3<T>& b) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = a.e[i][0] * b.e[0][j] + a.e[i][1] * b.e[1][j] + a.e[i][2] * b.e[2][j];
    return r;
}
// rows 0, 1 of a^+ b
template <class T> __device__ __forceinline__ M3<T> mul_dn_2(const M3<T>& a, const M3<T>& b) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            r.e[i][j] = mulc(b.e[0][j], a.e[0][i]) + mulc(b.e[1][j], a.e[1][i]) + mulc(b.e[2][j], a.e[2][i]);
    return r;
}

template <> __device__ __forceinline__ M3<float> mul_nd_2<float>(const M3<float>& a, const M3<float>& b) {
    return x2_product<2, false, true>(a, b);
}
template <> __device__ __forceinline__ M3<float> mul_nn_2<float>(const M3<float>& a, const M3<float>& b) {
    return x2_product<2, false, false>(a, b);
}
template <> __device__ __forceinline__ M3<float> mul_dn_2<float>(const M3<float>& a, const M3<float>& b) {
    return x2_product<2, true, false>(a, b);
}

// =============================================================== staple
// A_mu(x) = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
//                          + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) ]
// so that Re Tr(U_mu(x) A_mu(x)) sums the six plaquettes holding U_mu(x).
// x has parity par; x +- e_nu has parity 1 - par, x + e_mu - e_nu parity par.
//
// Staple in two-row form (FP32 links, 12- or 18-real); each half-term is added to A
// as it completes (A += up, A += dn), the order of staple_staged, so that staged and
// unstaged kernels agree bit for bit.  Each staple term is a product of three
// SU(3) links, hence in SU(3): only rows 0, 1 of every partial product are
// computed and row 2 is rebuilt, and a link that enters only through its rows
// (the left factor) is never completed.
//   up = (a b^+) c^+            a = U_nu(x+mu), b = U_mu(x+nu), c = U_nu(x)
//   dn = (e d)^+ f              d = U_nu(x+mu-nu), e = U_mu(x-nu), f = U_nu(x-nu)
template <class T, class LinkField>
__device__ __forceinline__ M3<T> staple_two_row(const LinkField& U, const Geom& g, const int x[4], int h, int mu,
                                                int par) {
    M3<T> A;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) A.e[i][j] = mk(T(0), T(0));
    const int op = par ^ 1;
    const Hops H = make_hops(g, x);
    const int fmu = pick(H.fwd, mu);
    const int hpm = (H.lex + fmu) >> 1;
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        const int hpn = (H.lex + H.fwd[nu]) >> 1;
        const int hmn = (H.lex + H.bwd[nu]) >> 1;
        const int hpm_mn = (H.lex + fmu + H.bwd[nu]) >> 1;
        M3<T> up, dn;
        {
            M3<T> t = mul_nd_2(U.load_rows(nu, op, hpm), U.load(mu, op, hpn));
            rebuild_row2(t);
            up = mul_nd_2(t, U.load(nu, par, h));
            rebuild_row2(up);
        }
        {
            M3<T> t = mul_nn_2(U.load_rows(mu, op, hmn), U.load(nu, par, hpm_mn));
            rebuild_row2(t);
            dn = mul_dn_2(t, U.load(nu, op, hmn));
            rebuild_row2(dn);
        }
        acc_add(A, up);
        acc_add(A, dn);
    }
    return A;
}

// ---- the two-row staple with its links staged through shared memory ----
// For FP32 12-real (paired) links.  The staple's six half-terms (the up and the
// down product of each direction nu != mu, in increasing nu) each need three
// links; the thread copies the links of half-term k+1 into its own
// shared-memory slots with cp.async while it computes half-term k from the
// other buffer, so those loads are in flight during the arithmetic without
// holding registers.  The updated link itself is staged with the first
// half-term and read back after the staple.  Each half-term is added to A as
// it completes (A += up, A += dn).  sm: (2 stages x 3 links + 1) x 3 pair-planes
// x STAGED_THREADS float4 (STAGED_SMEM bytes per block of STAGED_THREADS
// threads), each thread using its own column; the fixed block size keeps every
// slot address a constant offset from one base.  Single-lattice sub-sweeps use
// it from STAGED_MIN_VH links per launch on: below about a wave of blocks the
// serial half-term pipeline of each thread is not hidden by other warps.
constexpr int STAGED_THREADS = 128;
constexpr int STAGED_MIN_VH = 49152;
constexpr int STAGED_SMEM = (2 * 3 + 1) * 3 * 16 * STAGED_THREADS;

__device__ __forceinline__ void cp_async16(float4* smem, const float4* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(__cvta_generic_to_global(gmem)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// slot j of a stage (j = 0..2), or the updated link's slot (stage 2, j = 0)
__device__ __forceinline__ float4* staged_slot(float4* sm, int stage, int j, int k) {
    return sm + ((stage * 3 + j) * 3 + k) * STAGED_THREADS + threadIdx.x;
}
__device__ __forceinline__ void stage_link(float4* sm, int stage, int j, const Links<float, 6>& U, int mu, int par, int h) {
    const float4* q = reinterpret_cast<const float4*>(U.block(mu, par, h)) + (h & 31);
#pragma unroll
    for (int k = 0; k < 3; k++) cp_async16(staged_slot(sm, stage, j, k), q + (k << 5));
}
__device__ __forceinline__ M3<float> staged_rows(float4* sm, int stage, int j) {
    M3<float> m;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float4 v = *staged_slot(sm, stage, j, k);
        m.e[(2 * k) / 3][(2 * k) % 3] = mk(v.x, v.y);
        m.e[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(v.z, v.w);
    }
    return m;
}
__device__ __forceinline__ M3<float> staged_full(float4* sm, int stage, int j) {
    M3<float> m = staged_rows(sm, stage, j);
    rebuild_row2(m);
    return m;
}
// the updated link staged by thread col of the block (slot (2, 0)), with the
// row 2 that thread wrote into its free slot (0, 2)
__device__ __forceinline__ M3<float> own_full_of(float4* sm, int col) {
    M3<float> m;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float4 v = sm[((2 * 3 + 0) * 3 + k) * STAGED_THREADS + col];
        m.e[(2 * k) / 3][(2 * k) % 3] = mk(v.x, v.y);
        m.e[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(v.z, v.w);
    }
    const float4 r0 = sm[((0 * 3 + 2) * 3 + 0) * STAGED_THREADS + col];
    const float2 r1 = *reinterpret_cast<const float2*>(&sm[((0 * 3 + 2) * 3 + 1) * STAGED_THREADS + col]);
    m.e[2][0] = mk(r0.x, r0.y);
    m.e[2][1] = mk(r0.z, r0.w);
    m.e[2][2] = mk(r1.x, r1.y);
    return m;
}

// A = the staple of U_MU(x) (as staple_two_row, with the accumulation above);
// u = U_MU(x) (full, row 2 rebuilt).  MU may be a run-time direction; the
// sub-sweeps pass a compile-time one.
struct NoWork {
    __device__ void operator()() const {}
};
// early(): independent work that runs while the first loads are in flight.
template <class Work = NoWork>
__device__ __forceinline__ M3<float> staple_staged(const Links<float, 6>& U, const Geom& g, const int x[4], int h,
                                                   const int MU, int par, float4* sm, M3<float>& u,
                                                   Work early = Work()) {
    const int op = par ^ 1;
    const Hops H = make_hops(g, x);
    const int fmu = pick(H.fwd, MU);
    const int hpm = (H.lex + fmu) >> 1;
    int hpn[3], hmn[3], hpm_mn[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int nu = i < MU ? i : i + 1;
        hpn[i] = (H.lex + pick(H.fwd, nu)) >> 1;
        hmn[i] = (H.lex + pick(H.bwd, nu)) >> 1;
        hpm_mn[i] = (H.lex + fmu + pick(H.bwd, nu)) >> 1;
    }
    // half-term k: nu = the (k/2)-th direction other than MU; even k: up = (a b^+) c^+
    // with a = U_nu(x+mu), b = U_mu(x+nu), c = U_nu(x); odd k: dn = (e d)^+ f with
    // d = U_nu(x+mu-nu), e = U_mu(x-nu), f = U_nu(x-nu)
    auto issue = [&](int k, int stage) {
        const int i = k >> 1, nu = i < MU ? i : i + 1;
        if ((k & 1) == 0) {
            stage_link(sm, stage, 0, U, nu, op, hpm);
            stage_link(sm, stage, 1, U, MU, op, hpn[i]);
            stage_link(sm, stage, 2, U, nu, par, h);
        } else {
            stage_link(sm, stage, 0, U, nu, par, hpm_mn[i]);
            stage_link(sm, stage, 1, U, MU, op, hmn[i]);
            stage_link(sm, stage, 2, U, nu, op, hmn[i]);
        }
    };
    stage_link(sm, 2, 0, U, MU, par, h);  // the updated link, with the first half-term
    issue(0, 0);
    cp_async_commit();
    issue(1, 1);
    cp_async_commit();
    early();
    M3<float> A;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) A.e[i][j] = mk(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 6; k++) {
        if (k < 5) cp_async_wait<1>();
        else cp_async_wait<0>();
        const int st = k & 1;
        M3<float> term;
        if ((k & 1) == 0) {
            const M3<float> t = mul_nd_2(staged_rows(sm, st, 0), staged_full(sm, st, 1));
            term = mul_nd_2(t, staged_full(sm, st, 2));
        } else {
            M3<float> t = mul_nn_2(staged_rows(sm, st, 1), staged_full(sm, st, 0));
            rebuild_row2(t);
            term = mul_dn_2(t, staged_full(sm, st, 2));
        }
        rebuild_row2(term);
        acc_add(A, term);
        if (k + 2 < 6) {
            issue(k + 2, st);
            cp_async_commit();
        }
    }
    u = staged_full(sm, 2, 0);
    return A;
}

// Full products in the oracle's order (the FP64 parity path).
template <class T, int NP>
__device__ __forceinline__ M3<T> staple_full(const Links<T, NP>& U, const Geom& g, const int x[4], int h, int mu,
                                             int par) {
    M3<T> A;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) A.e[i][j] = mk(T(0), T(0));
    const int op = par ^ 1;
    const Hops H = make_hops(g, x);
    const int fmu = pick(H.fwd, mu);
    const int hpm = (H.lex + fmu) >> 1;
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        const int hpn = (H.lex + H.fwd[nu]) >> 1;
        const int hmn = (H.lex + H.bwd[nu]) >> 1;
        const int hpm_mn = (H.lex + fmu + H.bwd[nu]) >> 1;
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

// FP32 (both formats): products of SU(3) factors in two-row form; FP64: full
// products in the oracle's order.
template <class T, int NP>
__device__ __forceinline__ M3<T> staple(const Links<T, NP>& U, const Geom& g, const int x[4], int h, int mu, int par) {
    if constexpr (sizeof(T) == 4) return staple_two_row<T>(U, g, x, h, mu, par);
    else return staple_full(U, g, x, h, mu, par);
}

// =============================================================== plaquette
// Per site: sum over mu < nu < ND of Re Tr[U_mu(x) U_nu(x+mu) (U_nu(x) U_mu(x+nu))^+]
// (ND = 4: all six planes; ND = 3: the planes of directions 0, 1, 2).
template <class T, int NP, int ND = 4>
__device__ __forceinline__ double site_plaquettes(const Links<T, NP>& U, const Geom& g, int par, int h) {
    int x[4];
    cb_coords(g, par, h, x);
    const int op = par ^ 1;
    const Hops H = make_hops(g, x);
    double acc = 0.0;
#pragma unroll
    for (int mu = 0; mu < ND - 1; mu++) {
        const int hpm = (H.lex + H.fwd[mu]) >> 1;
        if constexpr (sizeof(T) == 4) {
            // FP32: a = U_mu(x) U_nu(x+mu) and b = U_nu(x) U_mu(x+nu) are in SU(3),
            // so rows 0, 1 of each suffice: with s_ij = row_i(a) . conj(row_j(b)),
            // Tr(a b^+) = s00 + s11 + conj(s00 s11 - s01 s10) (row 2 = conj(row0 x row1)
            // and the Binet-Cauchy identity for the cross products).
            const M3<T> umu = U.load_rows(mu, par, h);
#pragma unroll
            for (int nu = mu + 1; nu < ND; nu++) {
                const int hpn = (H.lex + H.fwd[nu]) >> 1;
                const M3<T> a = mul_nn_2(umu, U.load(nu, op, hpm));
                const M3<T> b = mul_nn_2(U.load_rows(nu, par, h), U.load(mu, op, hpn));
                Cx<T> sij[2][2];
#pragma unroll
                for (int i = 0; i < 2; i++)
#pragma unroll
                    for (int j = 0; j < 2; j++)
                        sij[i][j] = mulc(a.e[i][0], b.e[j][0]) + mulc(a.e[i][1], b.e[j][1]) + mulc(a.e[i][2], b.e[j][2]);
                const Cx<T> d = sij[0][0] * sij[1][1] - sij[0][1] * sij[1][0];
                acc += (double)(sij[0][0].re + sij[1][1].re + d.re);
            }
        } else {
            const M3<T> umu = U.load(mu, par, h);
#pragma unroll
            for (int nu = mu + 1; nu < ND; nu++) {
                const int hpn = (H.lex + H.fwd[nu]) >> 1;
                const M3<T> a = mul_nn(umu, U.load(nu, op, hpm));
                const M3<T> b = mul_nn(U.load(nu, par, h), U.load(mu, op, hpn));
                acc += (double)retr_nd(a, b);
            }
        }
    }
    return acc;
}

// =============================================================== clover
// Clover leaves around x in the (mu,nu) plane, all starting and ending at x,
// counterclockwise; returns the algebra coefficients g of
// G = traceless part of (Q - Q^+)/8, i.e. g = t(TA(Q))/4.
template <class T, int NP>
__device__ __forceinline__ void clover_coeffs(const Links<T, NP>& U, const Geom& g, const int x[4], int par, int h, int mu,
                                              int nu, T out[8]) {
    const int op = par ^ 1;
    const int lpm = lex_hop(g, x, mu, +1), lpn = lex_hop(g, x, nu, +1);
    const int lmm = lex_hop(g, x, mu, -1), lmn = lex_hop(g, x, nu, -1);
    const int lmm_pn = lex_hop(g, x, mu, -1, nu, +1);
    const int lmm_mn = lex_hop(g, x, mu, -1, nu, -1);
    const int lpm_mn = lex_hop(g, x, mu, +1, nu, -1);
    const M3<T> umu = U.load(mu, par, h), unu = U.load(nu, par, h);
    // l1 = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    M3<T> Q = mul_nd(mul_nn(umu, U.load(nu, op, lpm >> 1)), mul_nn(unu, U.load(mu, op, lpn >> 1)));
    // l2 = U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
    {
        const M3<T> a = U.load(mu, par, lmm_pn >> 1), b = U.load(nu, op, lmm >> 1), c = U.load(mu, op, lmm >> 1);
        acc_add(Q, mul_nn(mul_nd(unu, a), mul_dn(b, c)));
    }
    // l3 = U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
    {
        const M3<T> a = U.load(mu, op, lmm >> 1), b = U.load(nu, par, lmm_mn >> 1), c = U.load(mu, par, lmm_mn >> 1),
                    d = U.load(nu, op, lmn >> 1);
        acc_add(Q, mul_nn(mul_dd(a, b), mul_nn(c, d)));
    }
    // l4 = U_nu(x-nu)^+ U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^+
    {
        const M3<T> a = U.load(nu, op, lmn >> 1), b = U.load(mu, op, lmn >> 1), c = U.load(nu, par, lpm_mn >> 1);
        acc_add(Q, mul_nd(mul_nn(mul_dn(a, b), c), umu));
    }
    ta_coeffs(Q, out);
#pragma unroll
    for (int a = 0; a < 8; a++) out[a] *= T(0.25);
}

// =============================================================== SU(2) steps
// rows i, j of m <- R(r) rows i, j, restricted to the rows (do_i, do_j) and
// columns (bit masks ci, cj) that are read later; with the subgroup index a
// compile-time constant the unused updates vanish.
template <class T>
__device__ __forceinline__ void su2_rows(M3<T>& m, int i, int j, const T r[4], bool do_i, bool do_j, int ci, int cj) {
    const Cx<T> a = mk(r[0], r[3]), b = mk(r[2], r[1]), c = mk(-r[2], r[1]), d = mk(r[0], -r[3]);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const Cx<T> mi = m.e[i][k], mj = m.e[j][k];
        if (do_i && ((ci >> k) & 1)) m.e[i][k] = a * mi + b * mj;
        if (do_j && ((cj >> k) & 1)) m.e[j][k] = c * mi + d * mj;
    }
}

// FP32: a m_i + b m_j with a = r0 + i r3, b = r2 + i r1 (and c = -r2 + i r1,
// d = r0 - i r3 for row j) as packed FMAs on (re, im) pairs.
template <>
__device__ __forceinline__ void su2_rows<float>(M3<float>& m, int i, int j, const float r[4], bool do_i, bool do_j,
                                                int ci, int cj) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float2 MI = make_float2(m.e[i][k].re, m.e[i][k].im), iMI = make_float2(-m.e[i][k].im, m.e[i][k].re);
        const float2 MJ = make_float2(m.e[j][k].re, m.e[j][k].im), iMJ = make_float2(-m.e[j][k].im, m.e[j][k].re);
        if (do_i && ((ci >> k) & 1)) {
            float2 v = __fmul2_rn(bcast(r[0]), MI);
            v = __ffma2_rn(bcast(r[3]), iMI, v);
            v = __ffma2_rn(bcast(r[2]), MJ, v);
            v = __ffma2_rn(bcast(r[1]), iMJ, v);
            m.e[i][k] = from_f2(v);
        }
        if (do_j && ((cj >> k) & 1)) {
            float2 v = __fmul2_rn(bcast(-r[2]), MI);
            v = __ffma2_rn(bcast(r[1]), iMI, v);
            v = __ffma2_rn(bcast(r[0]), MJ, v);
            v = __ffma2_rn(bcast(-r[3]), iMJ, v);
            m.e[j][k] = from_f2(v);
        }
    }
}

// After the update of subgroup s: U needs rows 0, 1 (the final
// reunitarisation rebuilds row 2) and, until s = 2, row 2 as an input; V only
// needs the entries the later subgroups read (s = 1 reads row 0 and
// V20, V22, s = 2 reads V11, V12, V21, V22).
template <class T>
__device__ __forceinline__ void apply_subgroup(M3<T>& u, M3<T>& v, int s, const T R[4]) {
    if (s == 0) {
        su2_rows(u, 0, 1, R, true, true, 7, 7);
        su2_rows(v, 0, 1, R, true, true, 7, 6);
    } else if (s == 1) {
        su2_rows(u, 0, 2, R, true, true, 7, 7);
        su2_rows(v, 0, 2, R, false, true, 0, 6);
    } else {
        su2_rows(u, 1, 2, R, true, false, 7, 0);
    }
}

// Creutz's a0 and the direction (cos phi, sin phi), phi = 2 pi u3.  FP64 uses
// the accurate library functions (the oracle's operations); FP32 uses the
// hardware exponential, logarithm and sine/cosine where their absolute error
// (~1e-6) is harmless, and the accurate forms near their ill-conditioned ends.
__device__ __forceinline__ double creutz_a0(double k, double em, double u0) { return 1.0 + log1p((1.0 - u0) * em) / k; }
__device__ __forceinline__ float creutz_a0(float k, float em, float u0) {
    const float y = (1.f - u0) * em;
    return 1.f + (y < -0.1f ? __logf(1.f + y) : log1pf(y)) * __frcp_rn(k);
}
__device__ __forceinline__ double creutz_k(double beta, double xi) { return 2.0 * beta * xi / 3.0; }
__device__ __forceinline__ float creutz_k(float beta, float xi) { return xi * (beta * 0.666666667f); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
// sqrt of a positive argument (both uses above are > 0: rest >= u1^2 > 0 and
// |cos theta| < 1); FP32 takes x rsqrt(x)
__device__ __forceinline__ double sampler_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float sampler_sqrt(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double creutz_em(double k) { return expm1(-2.0 * k); }
__device__ __forceinline__ float creutz_em(float k) { return k > 0.25f ? __expf(-2.f * k) - 1.f : expm1f(-2.f * k); }
__device__ __forceinline__ void creutz_phi(double u3, double* s, double* c) { sincospi(2.0 * u3, s, c); }
__device__ __forceinline__ void creutz_phi(float u3, float* s, float* c) {
    // 2 pi u3 - pi lies in (-pi, pi), where __sincosf is accurate; shift back by pi
    float sn, cs;
    __sincosf(fmaf(6.28318530718f, u3, -3.14159265359f), &sn, &cs);
    *s = -sn;
    *c = -cs;
}

// =============================================================== heat bath
// One link: V = U A; per subgroup (0,1), (0,2), (1,2): w from the block,
// k = 2 beta |w| / 3, up to n_hb Creutz attempts
//   a0 = 1 + log1p((1 - u0) expm1(-2k)) / k, accept iff u1^2 <= 1 - a0^2,
// direction cos(theta) = 2 u2 - 1, phi = 2 pi u3; R = X (w/|w|), U <- R U,
// V <- R V; reunitarise at the end.  dec[s] = accepted attempt or 255.

// One Creutz attempt on subgroup s with the four words r; on acceptance
// applies R = X (w/|w|) to u and v and returns true.
template <class T>
__device__ __forceinline__ bool creutz_attempt(M3<T>& u, M3<T>& v, int s, const T w[4], T xi, T k, T em, uint4 r) {
    const T u0 = u01<T>(r.x), u1 = u01<T>(r.y), u2 = u01<T>(r.z), u3 = u01<T>(r.w);
    const T a0 = creutz_a0(k, em, u0);
    const T rest = sub_rn(T(1), mul_rn(a0, a0));
    if (!(mul_rn(u1, u1) <= rest)) return false;
    const T rad = sampler_sqrt(rest);
    const T ct = T(2) * u2 - T(1);
    const T st = sampler_sqrt(sub_rn(T(1), mul_rn(ct, ct)));
    T sp, cp;
    creutz_phi(u3, &sp, &cp);
    const T X[4] = {a0, rad * st * cp, rad * st * sp, rad * ct};
    const T inv = recip(xi);
    const T wh[4] = {w[0] * inv, w[1] * inv, w[2] * inv, w[3] * inv};
    T R[4];
    qmul(X, wh, R);
    apply_subgroup(u, v, s, R);
    return true;
}

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
            const T k = creutz_k(beta, xi);
            const T em = creutz_em(k);
            for (int att = 0; att < n_hb; att++) {
                if (creutz_attempt(u, v, s, w, xi, k, em, draw(rk, lex, mu, (uint32_t)s, (uint32_t)att, KIND_HB))) {
                    d = (uint8_t)att;
                    break;
                }
            }
        }
        if (dec) dec[s] = d;
    }
    reunitarize(u);
}

// The single-attempt heat bath with the three draws given (r[s]: subgroup s,
// attempt 0), so that a kernel can draw them while its loads are in flight.
template <class T>
__device__ __forceinline__ void hb_link_drawn(M3<T>& u, const M3<T>& A, T beta, const uint4 r[3]) {
    M3<T> v = mul_nn(u, A);
#pragma unroll
    for (int s = 0; s < 3; s++) {
        const int i = (s == 2) ? 1 : 0, j = (s == 0) ? 1 : 2;
        T w[4];
        block_w(v, i, j, w);
        const T xi = m_sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        if (xi >= tiny_norm<T>()) {
            const T k = creutz_k(beta, xi);
            creutz_attempt(u, v, s, w, xi, k, creutz_em(k), r[s]);
        }
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
        const T inv2 = recip(n2);
        // (w/|w|)^2 = (w0^2 - |w_vec|^2, 2 w0 w_vec) / |w|^2
        const T R[4] = {(w[0] * w[0] - w[1] * w[1] - w[2] * w[2] - w[3] * w[3]) * inv2, T(2) * w[0] * w[1] * inv2,
                        T(2) * w[0] * w[2] * inv2, T(2) * w[0] * w[3] * inv2};
        apply_subgroup(u, v, s, R);
    }
    reunitarize(u);
}

}  // namespace mgq
