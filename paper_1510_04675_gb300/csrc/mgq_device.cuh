// Device-side building blocks of libmgq: complex and 3x3 complex matrices,
// lattice geometry in the even/odd structure-of-arrays layout, link loads and
// stores (18-real and 12-real formats), Philox4x32-10, SU(2)/SU(3) algebra.
//
// Everything is templated on the arithmetic type T (double or float) so the
// FP64 parity path and the FP32 fast path are the same source.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mgq {

// ----------------------------------------------------------------- math shims
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double m_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_acos(float x) { return acosf(x); }
__device__ __forceinline__ double m_acos(double x) { return acos(x); }
__device__ __forceinline__ void m_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void m_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void m_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void m_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }
// products and differences that must not be contracted into an FMA (the
// accept/reject comparison is evaluated with separately rounded operations)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// |w| below which an SU(2) subgroup update is skipped
template <class T> __device__ __forceinline__ T tiny_norm();
template <> __device__ __forceinline__ double tiny_norm<double>() { return 1e-300; }
template <> __device__ __forceinline__ float tiny_norm<float>() { return 1e-30f; }

// ----------------------------------------------------------------- complex
template <class T>
struct alignas(2 * sizeof(T)) Cx {
    T re, im;
};

template <class T> __device__ __forceinline__ Cx<T> mk(T r, T i) { Cx<T> z; z.re = r; z.im = i; return z; }
template <class T> __device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <class T> __device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <class T> __device__ __forceinline__ Cx<T> operator*(Cx<T> a, Cx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T> __device__ __forceinline__ Cx<T> scale(Cx<T> a, T s) { return mk(a.re * s, a.im * s); }
template <class T> __device__ __forceinline__ Cx<T> conjg(Cx<T> a) { return mk(a.re, -a.im); }
// a * conj(b)
template <class T> __device__ __forceinline__ Cx<T> mulc(Cx<T> a, Cx<T> b) {
    return mk(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
template <class T> __device__ __forceinline__ T norm2(Cx<T> a) { return a.re * a.re + a.im * a.im; }

// ----------------------------------------------------------------- 3x3
template <class T>
struct M3 {
    Cx<T> e[3][3];
};

template <class T> __device__ __forceinline__ M3<T> unit3() {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = mk<T>(i == j ? T(1) : T(0), T(0));
    return r;
}

// a b
template <class T> __device__ __forceinline__ M3<T> mul_nn(const M3<T>& a, const M3<T>& b) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = a.e[i][0] * b.e[0][j] + a.e[i][1] * b.e[1][j] + a.e[i][2] * b.e[2][j];
    return r;
}
// a b^+
template <class T> __device__ __forceinline__ M3<T> mul_nd(const M3<T>& a, const M3<T>& b) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            r.e[i][j] = mulc(a.e[i][0], b.e[j][0]) + mulc(a.e[i][1], b.e[j][1]) + mulc(a.e[i][2], b.e[j][2]);
    return r;
}
// a^+ b
template <class T> __device__ __forceinline__ M3<T> mul_dn(const M3<T>& a, const M3<T>& b) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            r.e[i][j] = mulc(b.e[0][j], a.e[0][i]) + mulc(b.e[1][j], a.e[1][i]) + mulc(b.e[2][j], a.e[2][i]);
    return r;
}
// a^+ b^+ = (b a)^+
template <class T> __device__ __forceinline__ M3<T> mul_dd(const M3<T>& a, const M3<T>& b) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            r.e[i][j] = conjg(b.e[j][0] * a.e[0][i] + b.e[j][1] * a.e[1][i] + b.e[j][2] * a.e[2][i]);
    return r;
}
// FP32 products on the packed f32x2 FMA of sm_100+: a complex product is
// a.re * (b.re, b.im) + a.im * (-b.im, b.re), two paired FMAs instead of four.
// ROWS = 2 computes rows 0 and 1 of the result only; DA / DB take the
// conjugate transpose of a / b.
__device__ __forceinline__ float2 bcast(float x) { return make_float2(x, x); }
__device__ __forceinline__ Cx<float> from_f2(float2 z) { return mk(z.x, z.y); }

template <int ROWS, bool DA, bool DB>
__device__ __forceinline__ M3<float> x2_product(const M3<float>& a, const M3<float>& b) {
    float2 B[3][3], iB[3][3];  // B[k][j] = (b_kj or conj(b_jk)), iB = i B
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float re = DB ? b.e[j][k].re : b.e[k][j].re;
            const float im = DB ? -b.e[j][k].im : b.e[k][j].im;
            B[k][j] = make_float2(re, im);
            iB[k][j] = make_float2(-im, re);
        }
    M3<float> r;
#pragma unroll
    for (int i = 0; i < ROWS; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float are = DA ? a.e[k][i].re : a.e[i][k].re;
                const float aim = DA ? -a.e[k][i].im : a.e[i][k].im;
                acc = __ffma2_rn(bcast(are), B[k][j], acc);
                acc = __ffma2_rn(bcast(aim), iB[k][j], acc);
            }
            r.e[i][j] = from_f2(acc);
        }
    return r;
}

template <> __device__ __forceinline__ M3<float> mul_nn<float>(const M3<float>& a, const M3<float>& b) {
    return x2_product<3, false, false>(a, b);
}
template <> __device__ __forceinline__ M3<float> mul_nd<float>(const M3<float>& a, const M3<float>& b) {
    return x2_product<3, false, true>(a, b);
}
template <> __device__ __forceinline__ M3<float> mul_dn<float>(const M3<float>& a, const M3<float>& b) {
    return x2_product<3, true, false>(a, b);
}
template <> __device__ __forceinline__ M3<float> mul_dd<float>(const M3<float>& a, const M3<float>& b) {
    return x2_product<3, true, true>(a, b);
}

template <class T> __device__ __forceinline__ void acc_add(M3<T>& a, const M3<T>& b) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) a.e[i][j] = a.e[i][j] + b.e[i][j];
}
template <> __device__ __forceinline__ void acc_add<float>(M3<float>& a, const M3<float>& b) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            a.e[i][j] = from_f2(__fadd2_rn(make_float2(a.e[i][j].re, a.e[i][j].im), make_float2(b.e[i][j].re, b.e[i][j].im)));
}
template <class T> __device__ __forceinline__ M3<T> dagger(const M3<T>& a) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = conjg(a.e[j][i]);
    return r;
}
// Re Tr(a b)
template <class T> __device__ __forceinline__ T retr_nn(const M3<T>& a, const M3<T>& b) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) s += a.e[i][k].re * b.e[k][i].re - a.e[i][k].im * b.e[k][i].im;
    return s;
}
// Re Tr(a b^+)
template <class T> __device__ __forceinline__ T retr_nd(const M3<T>& a, const M3<T>& b) {
    T s = T(0);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) s += a.e[i][k].re * b.e[i][k].re + a.e[i][k].im * b.e[i][k].im;
    return s;
}

// Third row of an SU(3) matrix from its first two: conj(row0 x row1).
template <class T> __device__ __forceinline__ void rebuild_row2(M3<T>& u) {
    u.e[2][0] = conjg(u.e[0][1] * u.e[1][2] - u.e[0][2] * u.e[1][1]);
    u.e[2][1] = conjg(u.e[0][2] * u.e[1][0] - u.e[0][0] * u.e[1][2]);
    u.e[2][2] = conjg(u.e[0][0] * u.e[1][1] - u.e[0][1] * u.e[1][0]);
}

// FP32: conj(a b - c d) per entry on the packed FMA, row 1 entries paired.
template <> __device__ __forceinline__ void rebuild_row2<float>(M3<float>& u) {
    float2 B[3], iB[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        B[k] = make_float2(u.e[1][k].re, u.e[1][k].im);
        iB[k] = make_float2(-u.e[1][k].im, u.e[1][k].re);
    }
    // entry k: row0[p] row1[q] - row0[q] row1[p] with (p, q) = (1,2), (2,0), (0,1)
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int p = (k + 1) % 3, q = (k + 2) % 3;
        float2 acc = __fmul2_rn(bcast(u.e[0][p].re), B[q]);
        acc = __ffma2_rn(bcast(u.e[0][p].im), iB[q], acc);
        acc = __ffma2_rn(bcast(-u.e[0][q].re), B[p], acc);
        acc = __ffma2_rn(bcast(-u.e[0][q].im), iB[p], acc);
        u.e[2][k] = mk(acc.x, -acc.y);
    }
}

// 1/sqrt(n): the correctly rounded quotient in FP64 (the oracle's operations),
// the hardware reciprocal square root in FP32.
__device__ __forceinline__ double inv_norm(double n) { return 1.0 / sqrt(n); }
__device__ __forceinline__ float inv_norm(float n) { return rsqrtf(n); }

// Gram-Schmidt reunitarisation: normalise row 0, orthogonalise and
// normalise row 1, rebuild row 2 (determinant one).
template <class T> __device__ __forceinline__ void reunitarize(M3<T>& u) {
    T n0 = norm2(u.e[0][0]) + norm2(u.e[0][1]) + norm2(u.e[0][2]);
    T inv0 = inv_norm(n0);
#pragma unroll
    for (int k = 0; k < 3; k++) u.e[0][k] = scale(u.e[0][k], inv0);
    // <r0, row1> = sum conj(r0_k) row1_k
    Cx<T> ip = mulc(u.e[1][0], u.e[0][0]) + mulc(u.e[1][1], u.e[0][1]) + mulc(u.e[1][2], u.e[0][2]);
#pragma unroll
    for (int k = 0; k < 3; k++) u.e[1][k] = u.e[1][k] - ip * u.e[0][k];
    T n1 = norm2(u.e[1][0]) + norm2(u.e[1][1]) + norm2(u.e[1][2]);
    T inv1 = inv_norm(n1);
#pragma unroll
    for (int k = 0; k < 3; k++) u.e[1][k] = scale(u.e[1][k], inv1);
    rebuild_row2(u);
}

// ----------------------------------------------------------------- geometry
// Extents, volume, half volume and the padded per-parity site stride, with
// multiply-high constants for the divisions by L0, L1, L2 (set_divisors).
struct Geom {
    int L[4];
    int V, Vh, S;
    unsigned mg[3];
    int sh[3];
};

// Division by an invariant integer through a multiply-high (Granlund and
// Montgomery, PLDI 1994): for 2^(l-1) < L <= 2^l and m = ceil(2^(31+l) / L),
// floor(n / L) = floor(n m / 2^(31+l)) for every 0 <= n < 2^31; the product's
// high word shifted right by l - 1 gives it.  Site indices stay below 2^28.
inline void set_divisors(Geom& g) {
    for (int d = 0; d < 3; d++) {
        const unsigned long long L = (unsigned long long)g.L[d];
        int l = 0;
        while ((1ull << l) < L) l++;
        const unsigned long long p = 1ull << (31 + l);
        g.mg[d] = (unsigned)(p / L + (p % L ? 1 : 0));
        g.sh[d] = l - 1;
    }
}

__device__ __forceinline__ int div_L(const Geom& g, int d, int n) {
    return (int)(__umulhi((unsigned)n, g.mg[d]) >> g.sh[d]);
}

// Coordinates of checkerboard site (parity, h); h = lex/2.
__device__ __forceinline__ void cb_coords(const Geom& g, int par, int h, int x[4]) {
    const int lex2 = 2 * h;
    const int r0 = div_L(g, 0, lex2);
    const int x0e = lex2 - r0 * g.L[0];
    const int r1 = div_L(g, 1, r0);
    x[1] = r0 - r1 * g.L[1];
    x[3] = div_L(g, 2, r1);
    x[2] = r1 - x[3] * g.L[2];
    x[0] = x0e + ((par ^ (x[1] + x[2] + x[3])) & 1);
}

__device__ __forceinline__ int lex_of(const Geom& g, const int x[4]) {
    return x[0] + g.L[0] * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3]));
}

__device__ __forceinline__ int wrap(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// Lexicographic offsets of the neighbours of x, wrap-around included:
// lex(x + e_d) = lex + fwd[d], lex(x - e_d) = lex + bwd[d]; offsets of
// different directions add (lex(x + e_mu - e_nu) = lex + fwd[mu] + bwd[nu]).
struct Hops {
    int lex;
    int fwd[4], bwd[4];
};

__device__ __forceinline__ Hops make_hops(const Geom& g, const int x[4]) {
    Hops H;
    int st = 1;
#pragma unroll
    for (int d = 0; d < 4; d++) {
        H.fwd[d] = (x[d] == g.L[d] - 1) ? -(g.L[d] - 1) * st : st;
        H.bwd[d] = (x[d] == 0) ? (g.L[d] - 1) * st : -st;
        st *= g.L[d];
    }
    H.lex = lex_of(g, x);
    return H;
}

// a[d] for a run-time d without dynamic indexing (keeps a[] in registers)
__device__ __forceinline__ int pick(const int a[4], int d) { return d == 0 ? a[0] : d == 1 ? a[1] : d == 2 ? a[2] : a[3]; }

// Lexicographic index of x + dmu e_mu + dnu e_nu (|d| <= 1, periodic).
// Written with compile-time array indices only, so that a run-time mu or nu
// does not push the coordinates into local memory.
__device__ __forceinline__ int lex_hop(const Geom& g, const int x[4], int mu, int dmu, int nu = 0, int dnu = 0) {
    int y[4];
#pragma unroll
    for (int d = 0; d < 4; d++) y[d] = wrap(x[d] + (d == mu ? dmu : 0) + (d == nu ? dnu : 0), g.L[d]);
    return lex_of(g, y);
}

// ----------------------------------------------------------------- launch overlap
// Programmatic dependent launch: a sub-sweep launched with the programmatic
// stream-serialisation attribute may start while the previous kernel drains;
// it lets its own successor start likewise, does its index arithmetic, and
// waits for the previous kernel's completion (and memory) before it reads
// any link.  Without the attribute both instructions do nothing.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ----------------------------------------------------------------- fields
// load of one complex element.  A plain (coherent) global load, not the
// read-only path: kernels launched with programmatic dependent launch start
// before their predecessor has finished writing the links, and the
// read-only path is specified only for data that no one writes during the
// reading kernel's lifetime; the plain load after griddepcontrol.wait is
// ordered after those writes by the memory model.
__device__ __forceinline__ Cx<double> ldg_cx(const Cx<double>* p) {
    double2 v = *reinterpret_cast<const double2*>(p);
    return mk(v.x, v.y);
}
__device__ __forceinline__ Cx<float> ldg_cx(const Cx<float>* p) {
    float2 v = *reinterpret_cast<const float2*>(p);
    return mk(v.x, v.y);
}

// Link field: for each (mu, parity) the sites h = 0..S-1 come in blocks of 32
// consecutive h; a block holds plane 0 of its 32 sites, then plane 1, ...,
// i.e. links[mu][parity][h/32][plane][h%32].  NP = 9 planes (full matrix) or
// 6 (rows 0 and 1; row 2 rebuilt on load).  A warp reading one plane of 32
// consecutive sites reads 256 contiguous bytes, and the planes of one link sit
// at fixed 256-byte (FP32) steps, so a link costs one address computation.
// FP32 12-real links pair the planes instead: a block holds the pair-planes
// (0,1), (2,3), (4,5), each 32 sites x 16 bytes (re, im of plane 2p, then of
// plane 2p+1), i.e. links[mu][parity][h/32][pair][h%32][4 floats]: a link is
// three 16-byte loads, a warp's pair-plane 512 contiguous bytes.
template <class T, int NP>
struct Links {
    Cx<T>* p;
    int S;  // sites per (mu, parity), a multiple of 64
    static constexpr bool kPaired = sizeof(T) == 4 && NP == 6;

    // first element of the 32-site block holding h
    __device__ __forceinline__ Cx<T>* block(int mu, int par, int h) const {
        return p + ((size_t)((mu * 2 + par) * (S >> 5) + (h >> 5)) * NP << 5);
    }
    __device__ __forceinline__ Cx<T>* base(int mu, int par, int h) const { return block(mu, par, h) + (h & 31); }
    // the six planes of a paired link: three 16-byte loads
    __device__ __forceinline__ void load_pairs(int mu, int par, int h, M3<T>& m) const {
        const float4* q = reinterpret_cast<const float4*>(block(mu, par, h)) + (h & 31);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float4 v = q[k << 5];
            m.e[(2 * k) / 3][(2 * k) % 3] = mk(v.x, v.y);
            m.e[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(v.z, v.w);
        }
    }
    __device__ __forceinline__ M3<T> load(int mu, int par, int h) const {
        M3<T> m;
        if constexpr (kPaired) {
            load_pairs(mu, par, h, m);
        } else {
            const Cx<T>* b = base(mu, par, h);
#pragma unroll
            for (int r = 0; r < NP / 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) m.e[r][c] = ldg_cx(b + ((r * 3 + c) << 5));
        }
        if (NP == 6) rebuild_row2(m);
        return m;
    }
    // rows 0 and 1 only (row 2 left unset), for factors whose third row is not read
    __device__ __forceinline__ M3<T> load_rows(int mu, int par, int h) const {
        M3<T> m;
        if constexpr (kPaired) {
            load_pairs(mu, par, h, m);
        } else {
            const Cx<T>* b = base(mu, par, h);
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) m.e[r][c] = ldg_cx(b + ((r * 3 + c) << 5));
        }
        return m;
    }
    // load of a link given its lexicographic site (parity from the site)
    __device__ __forceinline__ M3<T> load_lex(int mu, int lex, int par) const { return load(mu, par, lex >> 1); }
    __device__ __forceinline__ void store(int mu, int par, int h, const M3<T>& m) const {
        if constexpr (kPaired) {
            float4* q = reinterpret_cast<float4*>(block(mu, par, h)) + (h & 31);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const Cx<T> a = m.e[(2 * k) / 3][(2 * k) % 3], b = m.e[(2 * k + 1) / 3][(2 * k + 1) % 3];
                q[k << 5] = make_float4(a.re, a.im, b.re, b.im);
            }
        } else {
            Cx<T>* b = base(mu, par, h);
#pragma unroll
            for (int r = 0; r < NP / 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) b[(r * 3 + c) << 5] = m.e[r][c];
        }
    }
};

// Lie-algebra field (8 reals per link) in the link field's block layout:
// alg[mu][parity][h/32][a][h%32].
template <class T>
struct Alg {
    T* p;
    int S;  // sites per (mu, parity), a multiple of 64
    static constexpr int kStep = 32;  // distance between coefficients a and a+1 of one link

    __device__ __forceinline__ T* at(int mu, int par, int h) const {
        return p + ((size_t)((mu * 2 + par) * (S >> 5) + (h >> 5)) * 8 << 5) + (h & 31);
    }
    __device__ __forceinline__ void load(int mu, int par, int h, T a[8]) const {
        const T* b = at(mu, par, h);
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = b[k * kStep];
    }
    __device__ __forceinline__ void store(int mu, int par, int h, const T a[8]) const {
        T* b = at(mu, par, h);
#pragma unroll
        for (int k = 0; k < 8; k++) b[k * kStep] = a[k];
    }
};

// ----------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, two
// 32x32->64 products per round, Weyl key schedule.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

enum : uint32_t { KIND_HB = 1, KIND_HOT = 2, KIND_MOM = 3, KIND_ACCEPT = 4 };

struct RngKey {
    uint2 key;       // (lo32(seed), hi32(seed) ^ lattice_id)
    uint32_t idx_lo, idx_hi;  // sweep or trajectory index
};

__host__ __device__ inline RngKey make_rng(uint64_t seed, uint32_t lattice_id, uint64_t index) {
    RngKey r;
    r.key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ lattice_id);
    r.idx_lo = (uint32_t)(index & 0xffffffffu);
    r.idx_hi = (uint32_t)(index >> 32);
    return r;
}

__device__ __forceinline__ uint4 draw(const RngKey& k, uint32_t lex, uint32_t mu, uint32_t sub, uint32_t att, uint32_t kind) {
    return philox(make_uint4(lex, mu | (sub << 2) | (att << 4) | (kind << 12), k.idx_lo, k.idx_hi), k.key);
}

// 32-bit word -> uniform in (0,1): exact (w + 1/2) 2^-32 in FP64; in FP32 the
// top 23 bits, (w>>9 + 1/2) 2^-23, also exact.
template <class T> __device__ __forceinline__ T u01(uint32_t w);
template <> __device__ __forceinline__ double u01<double>(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }
template <> __device__ __forceinline__ float u01<float>(uint32_t w) {
    // 1 + m 2^-23 built from the bits, minus (1 - 2^-24): exact (Sterbenz),
    // equal to (m + 1/2) 2^-23 with m = w >> 9, without an int-to-float conversion
    return __int_as_float(0x3f800000u | (w >> 9)) - 0x1.fffffep-1f;
}

// ----------------------------------------------------------------- su(3)
// Coefficients t_a of TA(M) = (M - M^+)/2 - Tr(...)/3 in the basis
// X_a = i lambda_a / 2 (so TA(M) = sum_a t_a X_a).
template <class T> __device__ __forceinline__ void ta_coeffs(const M3<T>& m, T t[8]) {
    const T inv_sqrt3 = T(0.57735026918962576451);
    t[0] = m.e[0][1].im + m.e[1][0].im;
    t[1] = m.e[0][1].re - m.e[1][0].re;
    t[2] = m.e[0][0].im - m.e[1][1].im;
    t[3] = m.e[0][2].im + m.e[2][0].im;
    t[4] = m.e[0][2].re - m.e[2][0].re;
    t[5] = m.e[1][2].im + m.e[2][1].im;
    t[6] = m.e[1][2].re - m.e[2][1].re;
    t[7] = (m.e[0][0].im + m.e[1][1].im - T(2) * m.e[2][2].im) * inv_sqrt3;
}

// Hermitian traceless Q = (1/2) sum_a c_a lambda_a, so that sum_a c_a X_a = i Q.
template <class T> __device__ __forceinline__ M3<T> herm_from_coeffs(const T c[8]) {
    const T inv_sqrt3 = T(0.57735026918962576451);
    const T h = T(0.5);
    M3<T> q;
    q.e[0][0] = mk(h * (c[2] + c[7] * inv_sqrt3), T(0));
    q.e[1][1] = mk(h * (-c[2] + c[7] * inv_sqrt3), T(0));
    q.e[2][2] = mk(-c[7] * inv_sqrt3, T(0));
    q.e[0][1] = mk(h * c[0], -h * c[1]);
    q.e[1][0] = mk(h * c[0], h * c[1]);
    q.e[0][2] = mk(h * c[3], -h * c[4]);
    q.e[2][0] = mk(h * c[3], h * c[4]);
    q.e[1][2] = mk(h * c[5], -h * c[6]);
    q.e[2][1] = mk(h * c[5], h * c[6]);
    return q;
}

// exp(i Q) for hermitian traceless Q by the Cayley-Hamilton form
// f0 + f1 Q + f2 Q^2 (Morningstar & Peardon, Phys. Rev. D 69 (2004) 054501):
// c0 = det Q, c1 = Tr(Q^2)/2, theta = arccos(c0/c0max), u = sqrt(c1/3) cos(theta/3),
// w = sqrt(c1) sin(theta/3); negative c0 handled by f_j(-c0) = (-1)^j conj(f_j(c0)).
template <class T> __device__ __forceinline__ M3<T> exp_iQ(const M3<T>& Q) {
    M3<T> Q2 = mul_nn(Q, Q);
    T c1 = T(0.5) * (Q2.e[0][0].re + Q2.e[1][1].re + Q2.e[2][2].re);
    // det Q = Tr(Q^3)/3 = Re Tr(Q Q2)/3
    T c0 = retr_nn(Q, Q2) / T(3);
    Cx<T> f0, f1, f2;
    if (c1 <= T(0)) {
        return unit3<T>();
    }
    const bool neg = c0 < T(0);
    T c0a = neg ? -c0 : c0;
    T s = m_sqrt(c1 / T(3));
    T c0max = T(2) * s * s * s;
    T ratio = c0a / c0max;
    ratio = ratio > T(1) ? T(1) : ratio;
    T theta = m_acos(ratio);
    T st, ct;
    m_sincos(theta / T(3), &st, &ct);
    T u = s * ct;
    T w = m_sqrt(c1) * st;
    T u2 = u * u, w2 = w * w;
    // xi0(w) = sin(w)/w and cos(w); short series near w = 0
    T xi0, cw;
    if (w2 < T(0.0025)) {
        xi0 = T(1) - w2 / T(6) * (T(1) - w2 / T(20) * (T(1) - w2 / T(42)));
        cw = T(1) - w2 / T(2) * (T(1) - w2 / T(12) * (T(1) - w2 / T(30)));
    } else {
        T sw;
        m_sincos(w, &sw, &cw);
        xi0 = sw / w;
    }
    T s2u, c2u, su, cu;
    m_sincos(T(2) * u, &s2u, &c2u);
    m_sincos(u, &su, &cu);
    Cx<T> e2iu = mk(c2u, s2u);
    Cx<T> emiu = mk(cu, -su);
    Cx<T> h0 = scale(e2iu, u2 - w2) + emiu * mk(T(8) * u2 * cw, T(2) * u * (T(3) * u2 + w2) * xi0);
    Cx<T> h1 = scale(e2iu, T(2) * u) - emiu * mk(T(2) * u * cw, -(T(3) * u2 - w2) * xi0);
    Cx<T> h2 = e2iu - emiu * mk(cw, T(3) * u * xi0);
    T inv = T(1) / (T(9) * u2 - w2);
    f0 = scale(h0, inv);
    f1 = scale(h1, inv);
    f2 = scale(h2, inv);
    if (neg) {
        f0 = conjg(f0);
        f1 = mk(-f1.re, f1.im);
        f2 = conjg(f2);
    }
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            Cx<T> v = f1 * Q.e[i][j] + f2 * Q2.e[i][j];
            if (i == j) v = v + f0;
            r.e[i][j] = v;
        }
    return r;
}

// exp(sum_a c_a X_a) for real coefficients c_a.
template <class T> __device__ __forceinline__ M3<T> exp_alg(const T c[8]) { return exp_iQ(herm_from_coeffs(c)); }

// ----------------------------------------------------------------- SU(2)
// Quaternion a <-> 2x2 matrix R(a) = [[a0 + i a3, a2 + i a1], [-a2 + i a1, a0 - i a3]].
// w of the (i,j) block of V satisfies Re Tr(R(a) Vblock) = 2 a.w.
template <class T> __device__ __forceinline__ void block_w(const M3<T>& v, int i, int j, T w[4]) {
    w[0] = T(0.5) * (v.e[i][i].re + v.e[j][j].re);
    w[1] = T(-0.5) * (v.e[i][j].im + v.e[j][i].im);
    w[2] = T(0.5) * (v.e[j][i].re - v.e[i][j].re);
    w[3] = T(0.5) * (v.e[j][j].im - v.e[i][i].im);
}

// rows i, j of m <- R(r) applied from the left
template <class T> __device__ __forceinline__ void left_su2(M3<T>& m, int i, int j, const T r[4]) {
    const Cx<T> a = mk(r[0], r[3]), b = mk(r[2], r[1]), c = mk(-r[2], r[1]), d = mk(r[0], -r[3]);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        Cx<T> mi = m.e[i][k], mj = m.e[j][k];
        m.e[i][k] = a * mi + b * mj;
        m.e[j][k] = c * mi + d * mj;
    }
}

// quaternion product c = a b  (R(c) = R(a) R(b))
template <class T> __device__ __forceinline__ void qmul(const T a[4], const T b[4], T c[4]) {
    c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    c[1] = a[0] * b[1] + b[0] * a[1] - (a[2] * b[3] - a[3] * b[2]);
    c[2] = a[0] * b[2] + b[0] * a[2] - (a[3] * b[1] - a[1] * b[3]);
    c[3] = a[0] * b[3] + b[0] * a[3] - (a[1] * b[2] - a[2] * b[1]);
}

}  // namespace mgq
