// libmgq: gradients of the clover energy density E and charge Q (Sec. IV.B-C)
// with respect to the links, for the backward pass of flowed clover
// observables (the cotangent that the adjoint flow then pulls back).
//
// With g_p(x) = t(TA(Q_p(x)))/4 the algebra coefficients of the clover field
// strength of plane p at x (Q_p the four leaves), an observable O(g) has
// dO = sum_{x,p} c_p(x) . dg_p(x), c = dO/dg:
//   E = (1/V) sum_x 1/2 sum_p |g_p|^2           -> c_p = g_p / V
//   Q = 1/(8 pi^2) sum_x (g01.g23 - g02.g13 + g03.g12) -> c01 = g23/(8 pi^2), ...
// and dg = t(TA(dQ))/4, c . t(TA(N)) = -2 Re Tr(C N) (C = sum c_a X_a), so
// dO = -1/2 sum Re Tr(C_p(x) dQ_p(x)).  A leaf F1 F2 F3 F4 varied in factor k
// (F_k = U_m or U_m^+, variation U_m -> exp(e) U_m) contributes to the link's
// cotangent +1/4 TA(F_k R_k) for an undaggered and -1/4 TA(R_k F_k) for a
// daggered factor, R_k = F_{k+1} .. F_4 C F_1 .. F_{k-1}.
#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

// plane index of (a, b), a < b: 01 02 03 12 13 23
__host__ __device__ constexpr int plane_of(int a, int b) { return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5); }

// clover leaves of plane (a, b) at x: factor j of leaf l is the link in
// direction (kDir ? b : a) at x + oa e_a + ob e_b, daggered if kDag
struct LeafFactor {
    int8_t dir_b, oa, ob, dag;
};
__constant__ LeafFactor c_leaves[4][4] = {
    {{0, 0, 0, 0}, {1, 1, 0, 0}, {0, 0, 1, 1}, {1, 0, 0, 1}},        // l1 = U_a(x) U_b(x+a) U_a(x+b)^+ U_b(x)^+
    {{1, 0, 0, 0}, {0, -1, 1, 1}, {1, -1, 0, 1}, {0, -1, 0, 0}},     // l2 = U_b(x) U_a(x-a+b)^+ U_b(x-a)^+ U_a(x-a)
    {{0, -1, 0, 1}, {1, -1, -1, 1}, {0, -1, -1, 0}, {1, 0, -1, 0}},  // l3 = U_a(x-a)^+ U_b(x-a-b)^+ U_a(x-a-b) U_b(x-b)
    {{1, 0, -1, 1}, {0, 0, -1, 0}, {1, 1, -1, 0}, {0, 0, 0, 1}},     // l4 = U_b(x-b)^+ U_a(x-b) U_b(x+a-b) U_a(x)^+
};

template <class T>
struct Planes6 {  // c_p(x): [p][parity][a][h] (scratch of this file only)
    T* p;
    int S;
    __device__ __forceinline__ T* at(int pl, int par, int h) const { return p + (size_t)(pl * 2 + par) * 8 * S + h; }
};

// Pass 1: c_p(x) for every site and plane.
template <class T, int NP>
__global__ void __launch_bounds__(128) k_clover_cotangent(Links<T, NP> U, Geom g, int obs, Planes6<T> C) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.V) return;
    const int par = idx >= g.Vh, h = idx - par * g.Vh;
    int x[4];
    cb_coords(g, par, h, x);
    T G[6][8];
    const int pl[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
#pragma unroll 1
    for (int p = 0; p < 6; p++) clover_coeffs(U, g, x, par, h, pl[p][0], pl[p][1], G[p]);
    const T invV = T(1) / (T)g.V, q = T(1.0 / (8.0 * 9.869604401089358));
#pragma unroll
    for (int p = 0; p < 6; p++) {
        T* out = C.at(p, par, h);
#pragma unroll
        for (int a = 0; a < 8; a++) {
            T v;
            if (obs == 0) v = G[p][a] * invV;
            else {
                // partner planes: 01<->23 (+), 02<->13 (-), 03<->12 (+)
                const int partner = 5 - p;
                const T sgn = (p == 1 || p == 4) ? T(-1) : T(1);
                v = sgn * q * G[partner][a];
            }
            out[(size_t)a * C.S] = v;
        }
    }
}

template <class T, int NP>
__device__ __forceinline__ M3<T> factor(const Links<T, NP>& U, const Geom& g, const int x[4], int a, int b,
                                        const LeafFactor& f) {
    int y[4];
#pragma unroll
    for (int d = 0; d < 4; d++) y[d] = wrap(x[d] + (d == a ? f.oa : 0) + (d == b ? f.ob : 0), g.L[d]);
    const int lex = lex_of(g, y);
    const M3<T> u = U.load(f.dir_b ? b : a, (y[0] + y[1] + y[2] + y[3]) & 1, lex >> 1);
    return f.dag ? dagger(u) : u;
}

// Pass 2: lam_m += scale * dO/de_m for every link m = U_rho(y).
template <class T, int NP>
__global__ void __launch_bounds__(128) k_clover_vjp(Links<T, NP> U, Geom g, Planes6<T> C, T scl, Alg<T> Lam) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * g.Vh) return;
    const int mp = idx / g.Vh, h = idx - mp * g.Vh, rho = mp >> 1, par = mp & 1;
    int y[4];
    cb_coords(g, par, h, y);
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 1
    for (int s = 0; s < 4; s++) {
        if (s == rho) continue;
        const int a = s < rho ? s : rho, b = s < rho ? rho : s;
        const int pl = plane_of(a, b);
        const bool rho_is_b = (rho == b);
#pragma unroll 1
        for (int l = 0; l < 4; l++) {
#pragma unroll 1
            for (int k = 0; k < 4; k++) {
                const LeafFactor fk = c_leaves[l][k];
                if ((fk.dir_b != 0) != rho_is_b) continue;
                // clover centre x with x + offset_k = y
                int x[4];
#pragma unroll
                for (int d = 0; d < 4; d++) x[d] = wrap(y[d] - (d == a ? fk.oa : 0) - (d == b ? fk.ob : 0), g.L[d]);
                const int xpar = (x[0] + x[1] + x[2] + x[3]) & 1;
                T c[8];
                const T* cp = C.at(pl, xpar, lex_of(g, x) >> 1);
#pragma unroll
                for (int q = 0; q < 8; q++) c[q] = cp[(size_t)q * C.S];
                const M3<T> cq = herm_from_coeffs(c);  // C = i Q
                M3<T> Cm;
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++) Cm.e[i][j] = mk(-cq.e[i][j].im, cq.e[i][j].re);
                // R_k = F_{k+1} .. F_4 C F_1 .. F_{k-1}
                M3<T> R = unit3<T>();
                for (int j = k + 1; j < 4; j++) R = mul_nn(R, factor(U, g, x, a, b, c_leaves[l][j]));
                R = mul_nn(R, Cm);
                for (int j = 0; j < k; j++) R = mul_nn(R, factor(U, g, x, a, b, c_leaves[l][j]));
                const M3<T> Fk = factor(U, g, x, a, b, fk);
                T t[8];
                if (!fk.dag) {
                    ta_coeffs(mul_nn(Fk, R), t);
#pragma unroll
                    for (int q = 0; q < 8; q++) acc[q] += T(0.25) * t[q];
                } else {
                    ta_coeffs(mul_nn(R, Fk), t);
#pragma unroll
                    for (int q = 0; q < 8; q++) acc[q] -= T(0.25) * t[q];
                }
            }
        }
    }
    T* out = Lam.at(rho, par, h);
#pragma unroll
    for (int q = 0; q < 8; q++) out[q * Alg<T>::kStep] += scl * acc[q];
}

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

uint64_t clover_vjp_scratch(const mgq_lattice* lat) {
    return round256(6ull * 2ull * 8ull * site_stride(lat->dims) * (lat->prec == MGQ_F64 ? 8 : 4));
}

}  // namespace mgq

using namespace mgq;

extern "C" {

uint64_t mgq_clover_vjp_scratch_bytes(const mgq_lattice* lat) {
    if (!lat || !links_bytes(lat)) return 0;
    return clover_vjp_scratch(lat);
}

mgq_status mgq_clover_vjp(const mgq_lattice* lat, int observable, double scale, void* lambda, void* scratch,
                          uint64_t scratch_bytes, void* stream) {
    Trace trace("mgq_clover_vjp");
    mgq_status s = check_lattice(lat, false, "mgq_clover_vjp");
    if (s) return s;
    if (observable != 0 && observable != 1) return fail(MGQ_EINVAL, "mgq_clover_vjp: observable must be 0 (E) or 1 (Q)");
    if (!lambda || ((uintptr_t)lambda & 15)) return fail(MGQ_EINVAL, "mgq_clover_vjp: lambda NULL or misaligned");
    if (!scratch || ((uintptr_t)scratch & 255)) return fail(MGQ_EINVAL, "mgq_clover_vjp: scratch NULL or not 256-byte aligned");
    if (scratch_bytes < clover_vjp_scratch(lat))
        return fail(MGQ_ENOMEM, "mgq_clover_vjp: scratch has %llu bytes, needs %llu", (unsigned long long)scratch_bytes,
                    (unsigned long long)clover_vjp_scratch(lat));
    const Geom g = make_geom(lat->dims);
    cudaStream_t st = as_stream(stream);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        Planes6<T> C;
        C.p = reinterpret_cast<T*>(scratch);
        C.S = g.S;
        k_clover_cotangent<T, NP><<<nblk(g.V, 128), 128, 0, st>>>(links_of<T, NP>(lat), g, observable, C);
        k_clover_vjp<T, NP><<<nblk(8L * g.Vh, 128), 128, 0, st>>>(links_of<T, NP>(lat), g, C, (T)scale,
                                                                   alg_at<T>(lambda, lat->dims));
    });
    return cuda_check("mgq_clover_vjp");
}

}  // extern "C"
