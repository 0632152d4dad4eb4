// libmgq adjoint of the Wilson flow (Sec. IV.B; reverse mode through the
// third-order Runge-Kutta step of Luscher's integrator).
//
// Cotangents are su(3) fields in algebra coefficients: a cotangent Lam at a
// field W pairs with a variation W_l -> exp(eps_l) W_l as sum_l Lam_l . eps_l
// (component dot product in the basis X_a = i lambda_a / 2, i.e. the inner
// product <A, B> = -2 Re Tr(A B)).
//
// One step W0 -> W3 with Z_i = eps Z(W_i), Z(W) = -TA(W A(W)):
//   X0 = Z0/4,                W1 = exp(X0) W0
//   X1 = 8/9 Z1 - 17/36 Z0,   W2 = exp(X1) W1
//   X2 = 3/4 Z2 - 8/9 Z1 + 17/36 Z0,   W3 = exp(X2) W2
// Reverse mode, given Lam at W3:
//   Xi2 = J(X2)* Lam;  Lam <- e^{-X2} Lam e^{X2};  Psi2 = 3/4 Xi2;                     Lam += eps DZ(W2)*[Psi2]
//   Xi1 = J(X1)* Lam;  Lam <- e^{-X1} Lam e^{X1};  Psi1 = 8/9 (Xi1 - Xi2);             Lam += eps DZ(W1)*[Psi1]
//   Xi0 = J(X0)* Lam;  Lam <- e^{-X0} Lam e^{X0};  Psi0 = Xi0/4 - 17/36 (Xi1 - Xi2);   Lam += eps DZ(W0)*[Psi0]
// with J(X)* = sum_n (-ad_X)^n / (n+1)!, the adjoint of the differential of
// exp (d/dt e^{X + tY} e^{-X} = sum_n ad_X^n Y / (n+1)!).
#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

mgq_status force_accumulate(const mgq_lattice* lat, void* B, double coef, double alpha, cudaStream_t st);
mgq_status exp_update(const mgq_lattice* lat, void* B, double s, cudaStream_t st);

// i Q for hermitian Q: the antihermitian matrix sum_a c_a X_a
template <class T> __device__ __forceinline__ M3<T> alg_matrix(const T c[8]) {
    const M3<T> q = herm_from_coeffs(c);
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = mk(-q.e[i][j].im, q.e[i][j].re);
    return r;
}

// [a, b] for antihermitian a, b: b a = (a b)^+, so [a, b] = a b - (a b)^+ from
// one product; the result is antihermitian entry by entry (r_ji = -conj(r_ij)
// exactly, the diagonal purely imaginary).
template <class T> __device__ __forceinline__ M3<T> commutator_ah(const M3<T>& a, const M3<T>& b) {
    const M3<T> ab = mul_nn(a, b);
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = ab.e[i][j] - conjg(ab.e[j][i]);
    return r;
}

// Per link: X = c0 Z0 + c1 Z1 + c2 Z2; Xi = J(X)* Lam, the series summed until a
// term drops below the precision's rounding of the partial sum (|X| is O(eps):
// a few terms; at most 12 in FP64 and 8 in FP32, enough for |X| <= 0.5);
// Lam <- e^{-X} Lam e^{X}.
template <class T>
__global__ void __launch_bounds__(128) k_dexp_adjoint(Geom g, Alg<T> Z0, Alg<T> Z1, Alg<T> Z2, T c0, T c1, T c2,
                                                      Alg<T> Lam, Alg<T> Xi) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * g.Vh) return;
    const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
    T z0[8], z1[8], z2[8], x[8], l[8];
    Z0.load(mu, par, h, z0);
    Z1.load(mu, par, h, z1);
    Z2.load(mu, par, h, z2);
    Lam.load(mu, par, h, l);
#pragma unroll
    for (int a = 0; a < 8; a++) x[a] = c0 * z0[a] + c1 * z1[a] + c2 * z2[a];
    const M3<T> X = alg_matrix(x);
    const M3<T> L = alg_matrix(l);
    M3<T> term = L, sum = L;
    const T tiny = sizeof(T) == 4 ? T(3e-8) : T(5e-17);
#pragma unroll 1
    for (int n = 1; n <= (sizeof(T) == 4 ? 8 : 12); n++) {
        term = commutator_ah(X, term);
        const T f = T(-1) / T(n + 1);
        T tmax = 0, smax = 0;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                term.e[i][j] = scale(term.e[i][j], f);
                sum.e[i][j] = sum.e[i][j] + term.e[i][j];
                tmax = fmax(tmax, fmax(fabs(term.e[i][j].re), fabs(term.e[i][j].im)));
                smax = fmax(smax, fmax(fabs(sum.e[i][j].re), fabs(sum.e[i][j].im)));
            }
        if (tmax <= tiny * smax) break;
    }
    T xi[8];
    ta_coeffs(sum, xi);
    Xi.store(mu, par, h, xi);
    const M3<T> E = exp_alg(x);
    const M3<T> Ln = mul_dn(E, mul_nn(L, E));
    T ln[8];
    ta_coeffs(Ln, ln);
    Lam.store(mu, par, h, ln);
}

// Per link: Gout = J(Om)* Gin = sum_n (-ad_Om)^n Gin / (n+1)!, the pull-back of a
// cotangent at exp(Om) U to the algebra variable Om.  The series runs until a
// term drops below the precision's rounding of the partial sum (at most 40
// terms), so it stays exact for |Om| of order one.  Gin and Gout may alias.
template <class T>
__global__ void __launch_bounds__(128) k_exp_vjp(Geom g, Alg<T> Om, Alg<T> Gin, Alg<T> Gout) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * g.Vh) return;
    const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
    T x[8], l[8];
    Om.load(mu, par, h, x);
    Gin.load(mu, par, h, l);
    const M3<T> X = alg_matrix(x);
    M3<T> term = alg_matrix(l), sum = term;
    const T tiny = sizeof(T) == 4 ? T(3e-8) : T(5e-17);
#pragma unroll 1
    for (int n = 1; n <= 40; n++) {
        term = commutator_ah(X, term);
        const T f = T(-1) / T(n + 1);
        T tmax = 0, smax = 0;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                term.e[i][j] = scale(term.e[i][j], f);
                sum.e[i][j] = sum.e[i][j] + term.e[i][j];
                tmax = fmax(tmax, fmax(fabs(term.e[i][j].re), fabs(term.e[i][j].im)));
                smax = fmax(smax, fmax(fabs(sum.e[i][j].re), fabs(sum.e[i][j].im)));
            }
        if (tmax <= tiny * smax) break;
    }
    T out[8];
    ta_coeffs(sum, out);
    Gout.store(mu, par, h, out);
}

// P <- a0 X0 + a1 X1 + a2 X2 (algebra coefficients, elementwise)
template <class T>
__global__ void k_alg_combine(Geom g, Alg<T> P, Alg<T> X0, Alg<T> X1, Alg<T> X2, T a0, T a1, T a2) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * g.Vh) return;
    const int mp = idx / g.Vh, h = idx - mp * g.Vh, mu = mp >> 1, par = mp & 1;
    T p[8], u[8], v[8], w[8];
    X0.load(mu, par, h, u);
    X1.load(mu, par, h, v);
    X2.load(mu, par, h, w);
#pragma unroll
    for (int a = 0; a < 8; a++) p[a] = a0 * u[a] + a1 * v[a] + a2 * w[a];
    P.store(mu, par, h, p);
}

template <class T, int NP>
__device__ __forceinline__ M3<T> psi_at(const Alg<T>& P, int mu, int par, int h) {
    T c[8];
    P.load(mu, par, h, c);
    return alg_matrix(c);
}

// Lam_m += scale * DZ(W)*[Psi]_m for every link m = U_rho(y).  Pairing Psi
// with Z gives sum_l Re Tr(Psi_l W_l A_l) up to a constant: every plaquette
// holding l, traced from l, with Psi_l in front of l.  Seen from one
// plaquette, a link it traverses forwards (as W) carries +Psi just before
// it, one it traverses backwards (as W^+) carries -Psi just after it.  Its
// cotangent at m is -TA(U_m R), R the rest of the loop after m with one
// insertion at a time, summed; the insertion at m itself is the self term
// -TA(W_m A_m Psi_m), which the two launches below add half by half (the upper
// and the lower staples of A_m).

template <class T> __device__ __forceinline__ M3<T> msub(const M3<T>& a, const M3<T>& b) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = a.e[i][j] - b.e[i][j];
    return r;
}

// The two plaquettes of plane (rho, nu) that hold m = U_rho(y), nu the K-th
// direction other than rho.  Traced from m:
//   up:   m X1 X2 X3,   X1 = U_nu(y+rho), X2 = U_rho(y+nu)^+, X3 = U_nu(y)^+
//         R_up = Psi_nu(y+rho) X1 X2 X3 - X1 X2 Psi_rho(y+nu) X3 - X1 X2 X3 Psi_nu(y)
//   down: m Y1 Y2 Y3,   Y1 = U_nu(y-nu+rho)^+, Y2 = U_rho(y-nu)^+, Y3 = U_nu(y-nu)
//         R_dn = -Y1 Psi_nu(y-nu+rho) Y2 Y3 - Y1 Y2 Psi_rho(y-nu) Y3 + Y1 Y2 Psi_nu(y-nu) Y3
// each summed by the product rule over the running prefix; SIDE 0 adds
// scale * (-TA(U_m (sum_nu R_up + A_up Psi_m))), SIDE 1 the same with R_dn and
// A_dn, A_up = sum_nu X1 X2 X3 and A_dn = sum_nu Y1 Y2 Y3 the two halves of the
// staple (one side per launch, directions in a rolled loop, keeps the live
// state in registers).  SIDE 0 folds X1 X2 X3 Psi_m into its last insertion
// (both Psi at y); SIDE 1 sums A_dn and multiplies by Psi_m once.
template <class T, int NP, int SIDE>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 1 : 4) k_flow_vjp_plane(Links<T, NP> U, Geom g, Alg<T> Psi, T scl, Alg<T> Lam) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * g.Vh) return;
    const int mp = idx / g.Vh, h = idx - mp * g.Vh, rho = mp >> 1, par = mp & 1;
    const int op = par ^ 1;
    int x[4];
    cb_coords(g, par, h, x);
    const Hops H = make_hops(g, x);
    const int frho = pick(H.fwd, rho);
    M3<T> Rs, As;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Rs.e[i][j] = As.e[i][j] = mk(T(0), T(0));
#pragma unroll 1
    for (int K = 0; K < 3; K++) {
    const int nu = K < rho ? K : K + 1;
    M3<T> R;
    if constexpr (SIDE == 0) {
        const int h_pr = (H.lex + frho) >> 1;             // y + rho  (op)
        const int h_pn = (H.lex + pick(H.fwd, nu)) >> 1;  // y + nu   (op)
        const M3<T> X1 = U.load(nu, op, h_pr);
        const M3<T> X2d = U.load(rho, op, h_pn);  // X2 = X2d^+
        const M3<T> X3d = U.load(nu, par, h);     // X3 = X3d^+
        const M3<T> P2 = mul_nd(X1, X2d);         // X1 X2
        const M3<T> S = mul_nd(P2, X3d);          // X1 X2 X3, the upper staple
        // the self term's X1 X2 X3 Psi_m joins the last insertion: - X1 X2 X3 (Psi_nu(y) - Psi_m)
        T cn[8], cm[8];
        Psi.load(nu, par, h, cn);
        Psi.load(rho, par, h, cm);
#pragma unroll
        for (int a = 0; a < 8; a++) cn[a] -= cm[a];
        // R_up + S Psi_m = Psi_nu(y+rho) S - (X1 X2 Psi_rho(y+nu)) X3 - S (Psi_nu(y) - Psi_m)
        R = msub(msub(mul_nn(psi_at<T, NP>(Psi, nu, op, h_pr), S),
                      mul_nd(mul_nn(P2, psi_at<T, NP>(Psi, rho, op, h_pn)), X3d)),
                 mul_nn(S, alg_matrix(cn)));
    } else {
        const int bnu = pick(H.bwd, nu);
        const int h_mn = (H.lex + bnu) >> 1;            // y - nu        (op)
        const int h_mn_pr = (H.lex + bnu + frho) >> 1;  // y - nu + rho  (par)
        const M3<T> Y1d = U.load(nu, par, h_mn_pr);  // Y1 = Y1d^+
        const M3<T> Y2d = U.load(rho, op, h_mn);     // Y2 = Y2d^+
        const M3<T> P2 = mul_dd(Y1d, Y2d);           // Y1 Y2
        // R_dn = (Y1 Y2 (Psi_c - Psi_b) - Y1 Psi_a Y2) Y3, Psi_b and Psi_c both at y - nu
        T cc[8], cb[8];
        Psi.load(nu, op, h_mn, cc);
        Psi.load(rho, op, h_mn, cb);
#pragma unroll
        for (int a = 0; a < 8; a++) cc[a] -= cb[a];
        const M3<T> Q = msub(mul_nn(P2, alg_matrix(cc)), mul_nd(mul_dn(Y1d, psi_at<T, NP>(Psi, nu, par, h_mn_pr)), Y2d));
        const M3<T> Y3 = U.load(nu, op, h_mn);
        R = mul_nn(Q, Y3);
        acc_add(As, mul_nn(P2, Y3));                 // Y1 Y2 Y3, the lower staple
    }
    acc_add(Rs, R);
    }
    if constexpr (SIDE == 1) acc_add(Rs, mul_nn(As, psi_at<T, NP>(Psi, rho, par, h)));  // the self term's half
    T t[8];
    ta_coeffs(mul_nn(U.load(rho, par, h), Rs), t);
    T* b = Lam.at(rho, par, h);
#pragma unroll
    for (int a = 0; a < 8; a++) b[a * Alg<T>::kStep] -= scl * t[a];
}

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

static mgq_status flow_vjp(const mgq_lattice* lat, const void* links, const void* psi, double scl, void* lam,
                           cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    dispatch_prec(lat->prec, [&]<class T, int NP>() {
        const Links<T, NP> W = links_at<T, NP>(const_cast<void*>(links), lat->dims);
        const Alg<T> P = alg_at<T>(const_cast<void*>(psi), lat->dims), L = alg_at<T>(lam, lat->dims);
        const int nb = nblk(8L * g.Vh, 128);
        k_flow_vjp_plane<T, NP, 0><<<nb, 128, 0, st>>>(W, g, P, (T)scl, L);
        k_flow_vjp_plane<T, NP, 1><<<nb, 128, 0, st>>>(W, g, P, (T)scl, L);
    });
    return cuda_check("flow_vjp");
}

static mgq_status dexp_adjoint(const mgq_lattice* lat, void* z0, void* z1, void* z2, double c0, double c1, double c2,
                               void* lam, void* xi, cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    if (lat->prec == MGQ_F64)
        k_dexp_adjoint<double><<<nblk(8L * g.Vh, 128), 128, 0, st>>>(
            g, alg_at<double>(z0, lat->dims), alg_at<double>(z1, lat->dims), alg_at<double>(z2, lat->dims), c0, c1, c2,
            alg_at<double>(lam, lat->dims), alg_at<double>(xi, lat->dims));
    else
        k_dexp_adjoint<float><<<nblk(8L * g.Vh, 128), 128, 0, st>>>(
            g, alg_at<float>(z0, lat->dims), alg_at<float>(z1, lat->dims), alg_at<float>(z2, lat->dims), (float)c0,
            (float)c1, (float)c2, alg_at<float>(lam, lat->dims), alg_at<float>(xi, lat->dims));
    return cuda_check("dexp_adjoint");
}

static mgq_status combine(const mgq_lattice* lat, void* p, void* x0, void* x1, void* x2, double a0, double a1,
                          double a2, cudaStream_t st) {
    const Geom g = make_geom(lat->dims);
    if (lat->prec == MGQ_F64)
        k_alg_combine<double><<<nblk(8L * g.Vh, 256), 256, 0, st>>>(
            g, alg_at<double>(p, lat->dims), alg_at<double>(x0, lat->dims), alg_at<double>(x1, lat->dims),
            alg_at<double>(x2, lat->dims), a0, a1, a2);
    else
        k_alg_combine<float><<<nblk(8L * g.Vh, 256), 256, 0, st>>>(
            g, alg_at<float>(p, lat->dims), alg_at<float>(x0, lat->dims), alg_at<float>(x1, lat->dims),
            alg_at<float>(x2, lat->dims), (float)a0, (float)a1, (float)a2);
    return cuda_check("combine");
}

uint64_t flow_adjoint_scratch(const mgq_lattice* lat) {
    return 2 * round256(links_bytes(lat)) + 7 * round256(alg_bytes(lat));
}

}  // namespace mgq

using namespace mgq;

extern "C" {

uint64_t mgq_flow_adjoint_scratch_bytes(const mgq_lattice* lat) {
    if (!lat || !links_bytes(lat)) return 0;
    return flow_adjoint_scratch(lat);
}

mgq_status mgq_flow_vjp(const mgq_lattice* lat, const void* psi, double scale, void* lambda, void* stream) {
    Trace trace("mgq_flow_vjp");
    mgq_status s = check_lattice(lat, false, "mgq_flow_vjp");
    if (s) return s;
    if (!psi || !lambda || ((uintptr_t)psi & 15) || ((uintptr_t)lambda & 15))
        return fail(MGQ_EINVAL, "mgq_flow_vjp: psi/lambda NULL or misaligned");
    return flow_vjp(lat, lat->links, psi, scale, lambda, as_stream(stream));
}

mgq_status mgq_wilson_flow_step_adjoint(const mgq_lattice* lat, double eps, void* lambda, void* scratch,
                                        uint64_t scratch_bytes, void* stream) {
    Trace trace("mgq_wilson_flow_step_adjoint");
    mgq_status s = check_lattice(lat, false, "mgq_wilson_flow_step_adjoint");
    if (s) return s;
    if (!(eps > 0.0)) return fail(MGQ_EINVAL, "mgq_wilson_flow_step_adjoint: eps must be > 0");
    if (!lambda || ((uintptr_t)lambda & 15)) return fail(MGQ_EINVAL, "mgq_wilson_flow_step_adjoint: lambda NULL or misaligned");
    if (!scratch || ((uintptr_t)scratch & 255)) return fail(MGQ_EINVAL, "mgq_wilson_flow_step_adjoint: scratch NULL or not 256-byte aligned");
    if (scratch_bytes < flow_adjoint_scratch(lat))
        return fail(MGQ_ENOMEM, "mgq_wilson_flow_step_adjoint: scratch has %llu bytes, needs %llu",
                    (unsigned long long)scratch_bytes, (unsigned long long)flow_adjoint_scratch(lat));
    cudaStream_t st = as_stream(stream);
    const uint64_t lb = round256(links_bytes(lat)), ab = round256(alg_bytes(lat));
    char* p = static_cast<char*>(scratch);
    void* W1 = p;
    void* W2 = p + lb;
    void* Z[3] = {p + 2 * lb, p + 2 * lb + ab, p + 2 * lb + 2 * ab};
    void* Xi[3] = {p + 2 * lb + 3 * ab, p + 2 * lb + 4 * ab, p + 2 * lb + 5 * ab};
    void* Psi = p + 2 * lb + 6 * ab;
    const uint64_t lbytes = links_bytes(lat);
    // forward recompute of the step from W0 = lat->links (left unchanged)
    mgq_lattice w = *lat;
    if ((s = force_accumulate(lat, Z[0], -eps, 0.0, st))) return s;  // Z0 = eps Z(W0)
    if (cudaMemcpyAsync(W1, lat->links, lbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return cuda_check("mgq_wilson_flow_step_adjoint");
    w.links = W1;
    if ((s = exp_update(&w, Z[0], 0.25, st))) return s;                   // W1 = exp(Z0/4) W0
    if ((s = force_accumulate(&w, Z[1], -eps, 0.0, st))) return s;        // Z1 = eps Z(W1)
    if (cudaMemcpyAsync(W2, W1, lbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return cuda_check("mgq_wilson_flow_step_adjoint");
    w.links = W2;
    if ((s = combine(lat, Psi, Z[0], Z[1], Z[1], -17.0 / 36.0, 8.0 / 9.0, 0.0, st))) return s;  // X1
    if ((s = exp_update(&w, Psi, 1.0, st))) return s;                     // W2 = exp(X1) W1
    if ((s = force_accumulate(&w, Z[2], -eps, 0.0, st))) return s;        // Z2 = eps Z(W2)
    // reverse stage 2
    if ((s = dexp_adjoint(lat, Z[0], Z[1], Z[2], 17.0 / 36.0, -8.0 / 9.0, 0.75, lambda, Xi[2], st))) return s;
    if ((s = combine(lat, Psi, Xi[2], Xi[2], Xi[2], 0.75, 0.0, 0.0, st))) return s;
    if ((s = flow_vjp(lat, W2, Psi, eps, lambda, st))) return s;
    // reverse stage 1
    if ((s = dexp_adjoint(lat, Z[0], Z[1], Z[2], -17.0 / 36.0, 8.0 / 9.0, 0.0, lambda, Xi[1], st))) return s;
    if ((s = combine(lat, Psi, Xi[1], Xi[2], Xi[2], 8.0 / 9.0, -8.0 / 9.0, 0.0, st))) return s;
    if ((s = flow_vjp(lat, W1, Psi, eps, lambda, st))) return s;
    // reverse stage 0
    if ((s = dexp_adjoint(lat, Z[0], Z[1], Z[2], 0.25, 0.0, 0.0, lambda, Xi[0], st))) return s;
    if ((s = combine(lat, Psi, Xi[0], Xi[1], Xi[2], 0.25, -17.0 / 36.0, 17.0 / 36.0, st))) return s;
    if ((s = flow_vjp(lat, lat->links, Psi, eps, lambda, st))) return s;
    return MGQ_OK;
}

mgq_status mgq_exp_vjp(const mgq_lattice* lat, const void* omega, const void* g_in, void* g_out, void* stream) {
    Trace trace("mgq_exp_vjp");
    mgq_status s = check_lattice(lat, false, "mgq_exp_vjp");
    if (s) return s;
    if (!omega || !g_in || !g_out || ((uintptr_t)omega & 15) || ((uintptr_t)g_in & 15) || ((uintptr_t)g_out & 15))
        return fail(MGQ_EINVAL, "mgq_exp_vjp: omega/g_in/g_out NULL or misaligned");
    cudaStream_t st = as_stream(stream);
    const Geom g = make_geom(lat->dims);
    void* om = const_cast<void*>(omega);
    void* gi = const_cast<void*>(g_in);
    if (lat->prec == MGQ_F64)
        k_exp_vjp<double><<<nblk(8L * g.Vh, 128), 128, 0, st>>>(g, alg_at<double>(om, lat->dims),
                                                               alg_at<double>(gi, lat->dims),
                                                               alg_at<double>(g_out, lat->dims));
    else
        k_exp_vjp<float><<<nblk(8L * g.Vh, 128), 128, 0, st>>>(g, alg_at<float>(om, lat->dims),
                                                              alg_at<float>(gi, lat->dims),
                                                              alg_at<float>(g_out, lat->dims));
    return cuda_check("mgq_exp_vjp");
}

}  // extern "C"
