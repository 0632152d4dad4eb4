/*
 * mgq oracle -- a plain, slow, FP64 CPU restatement of the data-parallel hot
 * path of "Multiscale Monte Carlo equilibration: Pure Yang-Mills theory"
 * (Endres, Brower, Detmold, Orginos, Pochinsky, arXiv:1510.04675).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library: everything here is written
 * out again from the paper and from the published methods it cites.
 *
 * Layout (the "canonical" layout, also used to exchange fields with the GPU
 * library): U[site][mu][row][col] as complex double, site = x0 + L0*(x1 +
 * L1*(x2 + L2*x3)) (x0 fastest), mu = 0..3.  Momenta / Lie-algebra fields
 * are P[site][mu][a], a = 0..7, coefficients of X_a = i*lambda_a/2.
 *
 * Every floating-point quantity is double.  Parallel loops (OpenMP) only
 * cover loops whose iterations are independent (one checkerboard subset,
 * one observable per site); every sum is taken sequentially in site order
 * afterwards, so results do not depend on the thread count.
 *
 * Parity status of each function is listed in its comment ("pinned by" /
 * "parity unpinned").
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;
typedef struct { cplx e[3][3]; } mat3;
typedef struct { int L[4]; long V; } lat_t;

/* RNG stream kinds (the "kind" field of the Philox counter). */
enum { KIND_HB = 1, KIND_HOT = 2, KIND_MOM = 3, KIND_ACCEPT = 4 };

static const double TWO_PI = 6.283185307179586;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications,   */
/* with the two-word key bumped by the Weyl constants between rounds.        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * One counter-based draw of four uniforms in (0,1).
 * counter = (site, mu | subgroup<<2 | attempt<<4 | kind<<12, lo32(sweep), hi32(sweep))
 * key     = (lo32(seed), hi32(seed) ^ lattice_id)
 * uniform = (w + 0.5) * 2^-32   (exact in double)
 */
static void draw4(uint64_t seed, uint32_t lattice_id, uint32_t site, int mu, int subgroup,
                  int attempt, int kind, uint64_t sweep, double u[4])
{
    uint32_t ctr[4], key[2], w[4];
    ctr[0] = site;
    ctr[1] = (uint32_t)mu | ((uint32_t)subgroup << 2) | ((uint32_t)attempt << 4) | ((uint32_t)kind << 12);
    ctr[2] = (uint32_t)(sweep & 0xffffffffu);
    ctr[3] = (uint32_t)(sweep >> 32);
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32) ^ lattice_id;
    orc_philox4x32_10(ctr, key, w);
    for (int i = 0; i < 4; i++) u[i] = ((double)w[i] + 0.5) * 0x1p-32;
}

/* Exposed for the tests: the four uniforms of one draw. */
void orc_draw_uniforms(uint64_t seed, uint32_t lattice_id, uint32_t site, int mu, int subgroup,
                       int attempt, int kind, uint64_t sweep, double* u)
{
    draw4(seed, lattice_id, site, mu, subgroup, attempt, kind, sweep, u);
}

/* Box-Muller: two unit normals from two uniforms. */
static void box_muller(double u0, double u1, double* g0, double* g1)
{
    double r = sqrt(-2.0 * log(u0));
    *g0 = r * cos(TWO_PI * u1);
    *g1 = r * sin(TWO_PI * u1);
}

/* ------------------------------------------------------------------------ */
/* Geometry: D = 4 hypercubic lattice with periodic boundary conditions      */
/* (Sec. III).                                                               */
/* ------------------------------------------------------------------------ */
static lat_t make_lat(const int* dims)
{
    lat_t g;
    g.V = 1;
    for (int mu = 0; mu < 4; mu++) { g.L[mu] = dims[mu]; g.V *= dims[mu]; }
    return g;
}

static void coords_of(const lat_t* g, long s, int x[4])
{
    for (int mu = 0; mu < 4; mu++) { x[mu] = (int)(s % g->L[mu]); s /= g->L[mu]; }
}

static long site_of(const lat_t* g, const int xin[4])
{
    long s = 0;
    for (int mu = 3; mu >= 0; mu--) {
        int xm = ((xin[mu] % g->L[mu]) + g->L[mu]) % g->L[mu];
        s = s * g->L[mu] + xm;
    }
    return s;
}

/* site s displaced by d lattice units along mu */
static long hop(const lat_t* g, long s, int mu, int d)
{
    int x[4];
    coords_of(g, s, x);
    x[mu] += d;
    return site_of(g, x);
}

static long hop2(const lat_t* g, long s, int mu, int dmu, int nu, int dnu)
{
    int x[4];
    coords_of(g, s, x);
    x[mu] += dmu;
    x[nu] += dnu;
    return site_of(g, x);
}

static int parity_of(const lat_t* g, long s)
{
    int x[4];
    coords_of(g, s, x);
    return (x[0] + x[1] + x[2] + x[3]) & 1;
}

/* ------------------------------------------------------------------------ */
/* 3x3 complex matrices                                                      */
/* ------------------------------------------------------------------------ */
static mat3 m_zero(void) { mat3 r; memset(&r, 0, sizeof r); return r; }
static mat3 m_unit(void) { mat3 r = m_zero(); for (int i = 0; i < 3; i++) r.e[i][i] = 1.0; return r; }

static mat3 m_mul(mat3 a, mat3 b)
{
    mat3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx acc = 0;
            for (int k = 0; k < 3; k++) acc += a.e[i][k] * b.e[k][j];
            r.e[i][j] = acc;
        }
    return r;
}

static mat3 m_dag(mat3 a)
{
    mat3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) r.e[i][j] = conj(a.e[j][i]);
    return r;
}

static mat3 m_add(mat3 a, mat3 b)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) a.e[i][j] += b.e[i][j];
    return a;
}

static mat3 m_sub(mat3 a, mat3 b)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) a.e[i][j] -= b.e[i][j];
    return a;
}

static mat3 m_scale(mat3 a, cplx s)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) a.e[i][j] *= s;
    return a;
}

static cplx m_trace(mat3 a) { return a.e[0][0] + a.e[1][1] + a.e[2][2]; }

static double m_frob(mat3 a)
{
    double s = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) s += creal(a.e[i][j] * conj(a.e[i][j]));
    return sqrt(s);
}

/* Link access in the canonical layout. */
static mat3 getU(const double* U, long s, int mu)
{
    mat3 r;
    memcpy(&r, U + ((size_t)s * 4 + mu) * 18, sizeof r);
    return r;
}

static void setU(double* U, long s, int mu, mat3 m)
{
    memcpy(U + ((size_t)s * 4 + mu) * 18, &m, sizeof m);
}

/*
 * Reunitarisation by Gram-Schmidt: normalise row 0, orthogonalise row 1
 * against it and normalise, then row 2 = conj(row0 x row1), which makes the
 * determinant one.  Pinned by: returns SU(3) to rounding; fixes SU(3)
 * matrices (tests/test_oracle_algebra.py).
 */
static mat3 reunit(mat3 m)
{
    mat3 r;
    double n0 = 0;
    for (int k = 0; k < 3; k++) n0 += creal(m.e[0][k] * conj(m.e[0][k]));
    n0 = sqrt(n0);
    for (int k = 0; k < 3; k++) r.e[0][k] = m.e[0][k] / n0;
    cplx ip = 0;
    for (int k = 0; k < 3; k++) ip += conj(r.e[0][k]) * m.e[1][k];
    for (int k = 0; k < 3; k++) r.e[1][k] = m.e[1][k] - ip * r.e[0][k];
    double n1 = 0;
    for (int k = 0; k < 3; k++) n1 += creal(r.e[1][k] * conj(r.e[1][k]));
    n1 = sqrt(n1);
    for (int k = 0; k < 3; k++) r.e[1][k] /= n1;
    r.e[2][0] = conj(r.e[0][1] * r.e[1][2] - r.e[0][2] * r.e[1][1]);
    r.e[2][1] = conj(r.e[0][2] * r.e[1][0] - r.e[0][0] * r.e[1][2]);
    r.e[2][2] = conj(r.e[0][0] * r.e[1][1] - r.e[0][1] * r.e[1][0]);
    return r;
}

/* ------------------------------------------------------------------------ */
/* SU(2) subgroups.  A unit quaternion a = (a0, a1, a2, a3) stands for the   */
/* 2x2 matrix R(a) = a0*1 + a1*e1 + a2*e2 + a3*e3 with e_k = i*sigma_k.      */
/* ------------------------------------------------------------------------ */
typedef struct { cplx e[2][2]; } mat2;

static mat2 quat_basis(int k)
{
    mat2 b;
    memset(&b, 0, sizeof b);
    switch (k) {
    case 0: b.e[0][0] = 1; b.e[1][1] = 1; break;                 /* 1          */
    case 1: b.e[0][1] = I; b.e[1][0] = I; break;                 /* i sigma_1  */
    case 2: b.e[0][1] = 1; b.e[1][0] = -1; break;                /* i sigma_2  */
    case 3: b.e[0][0] = I; b.e[1][1] = -I; break;                /* i sigma_3  */
    }
    return b;
}

static mat2 quat_to_mat(const double a[4])
{
    mat2 r;
    memset(&r, 0, sizeof r);
    for (int k = 0; k < 4; k++) {
        mat2 b = quat_basis(k);
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) r.e[i][j] += a[k] * b.e[i][j];
    }
    return r;
}

static mat2 m2_mul(mat2 a, mat2 b)
{
    mat2 r;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) r.e[i][j] = a.e[i][0] * b.e[0][j] + a.e[i][1] * b.e[1][j];
    return r;
}

/* Cabibbo-Marinari subgroup s acts on rows/columns (sub_i[s], sub_j[s]). */
static const int sub_i[3] = {0, 0, 1};
static const int sub_j[3] = {1, 2, 2};

/*
 * Projection of the (i,j) block W of V on the quaternion basis:
 * Re Tr(R(a) W) = 2 a.w  for every quaternion a, i.e. w_k = Re Tr(e_k W)/2.
 */
static void subgroup_w(mat3 V, int s, double w[4])
{
    int i = sub_i[s], j = sub_j[s];
    mat2 W;
    W.e[0][0] = V.e[i][i]; W.e[0][1] = V.e[i][j];
    W.e[1][0] = V.e[j][i]; W.e[1][1] = V.e[j][j];
    for (int k = 0; k < 4; k++) {
        mat2 prod = m2_mul(quat_basis(k), W);
        w[k] = 0.5 * creal(prod.e[0][0] + prod.e[1][1]);
    }
}

/* M <- R_embedded(s) * M : R acts on rows i, j. */
static mat3 embed_left(mat2 R, int s, mat3 M)
{
    int i = sub_i[s], j = sub_j[s];
    mat3 out = M;
    for (int c = 0; c < 3; c++) {
        out.e[i][c] = R.e[0][0] * M.e[i][c] + R.e[0][1] * M.e[j][c];
        out.e[j][c] = R.e[1][0] * M.e[i][c] + R.e[1][1] * M.e[j][c];
    }
    return out;
}

/* ------------------------------------------------------------------------ */
/* Staples, plaquette, Wilson action (Sec. III, Wilson action and loops).    */
/* ------------------------------------------------------------------------ */

/*
 * Staple sum A_mu(x) = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
 *                                     + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) ]
 * so that Re Tr(U_mu(x) A_mu(x)) is the sum of Re Tr over the six
 * plaquettes that contain U_mu(x).  Pinned by: sum_x,mu Re Tr(U A) equals
 * four times the plaquette sum (each plaquette has four links).
 */
static mat3 staple(const lat_t* g, const double* U, long s, int mu)
{
    mat3 A = m_zero();
    long xp = hop(g, s, mu, +1);
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        long xpn = hop(g, s, nu, +1);
        long xmn = hop(g, s, nu, -1);
        long xpm_mn = hop2(g, s, mu, +1, nu, -1);
        mat3 up = m_mul(m_mul(getU(U, xp, nu), m_dag(getU(U, xpn, mu))), m_dag(getU(U, s, nu)));
        mat3 dn = m_mul(m_mul(m_dag(getU(U, xpm_mn, nu)), m_dag(getU(U, xmn, mu))), getU(U, xmn, nu));
        A = m_add(A, m_add(up, dn));
    }
    return A;
}

/* Plaquette U_munu(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ */
static mat3 plaq_mat(const lat_t* g, const double* U, long s, int mu, int nu)
{
    long xpm = hop(g, s, mu, +1), xpn = hop(g, s, nu, +1);
    return m_mul(m_mul(getU(U, s, mu), getU(U, xpm, nu)),
                 m_mul(m_dag(getU(U, xpn, mu)), m_dag(getU(U, s, nu))));
}

/* Sum over the six mu<nu planes at site s of Re Tr U_munu(s). */
static double site_plaq_sum(const lat_t* g, const double* U, long s)
{
    double acc = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++) acc += creal(m_trace(plaq_mat(g, U, s, mu, nu)));
    return acc;
}

/*
 * Average plaquette  W^{1x1} = (1/N_2) sum_x sum_{mu<nu} (1/3) Re Tr U_munu(x),
 * N_2 = 6 V (Sec. III).  Pinned by: unit gauge gives 1; gauge invariance;
 * strong and weak coupling limits of the heat bath; constant abelian flux.
 */
double orc_plaquette(const double* U, const int* dims)
{
    lat_t g = make_lat(dims);
    double* part = malloc(sizeof(double) * g.V);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++) part[s] = site_plaq_sum(&g, U, s);
    double acc = 0;
    for (long s = 0; s < g.V; s++) acc += part[s];
    free(part);
    return acc / (3.0 * 6.0 * (double)g.V);
}

/* Wilson action S = beta sum_x sum_{mu<nu} [1 - (1/3) Re Tr U_munu(x)] (Sec. III). */
double orc_action(const double* U, const int* dims, double beta)
{
    lat_t g = make_lat(dims);
    double w = orc_plaquette(U, dims);
    return beta * 6.0 * (double)g.V * (1.0 - w);
}

/* Exposed for tests: staple of one link into A (18 doubles). */
void orc_staple(const double* U, const int* dims, long s, int mu, double* A)
{
    lat_t g = make_lat(dims);
    mat3 a = staple(&g, U, s, mu);
    memcpy(A, &a, sizeof a);
}

/* ------------------------------------------------------------------------ */
/* Start configurations (Sec. IV.E: cold = ordered, hot = random).           */
/* ------------------------------------------------------------------------ */
static mat3 haar_link(uint64_t seed, uint32_t lattice_id, long s, int mu)
{
    double gs[20];
    for (int call = 0; call < 5; call++) {
        double u[4];
        draw4(seed, lattice_id, (uint32_t)s, mu, 0, call, KIND_HOT, 0, u);
        box_muller(u[0], u[1], &gs[4 * call + 0], &gs[4 * call + 1]);
        box_muller(u[2], u[3], &gs[4 * call + 2], &gs[4 * call + 3]);
    }
    mat3 Z;
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) Z.e[r][c] = gs[2 * (3 * r + c)] + I * gs[2 * (3 * r + c) + 1];
    return reunit(Z);
}

/* start = 0: every link is the unit matrix; start = 1: Haar-random SU(3). */
void orc_init_links(double* U, const int* dims, int start, uint64_t seed, uint32_t lattice_id)
{
    lat_t g = make_lat(dims);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++)
        for (int mu = 0; mu < 4; mu++) setU(U, s, mu, start ? haar_link(seed, lattice_id, s, mu) : m_unit());
}

/* ------------------------------------------------------------------------ */
/* Cabibbo-Marinari heat bath with Creutz's SU(2) sampler, and               */
/* overrelaxation (Sec. IV.A).                                               */
/* ------------------------------------------------------------------------ */

/*
 * Creutz's sampler for the SU(2) weight exp(k a0) on the Haar measure:
 * a0 = 1 + log(exp(-2k) + (1 - exp(-2k)) v)/k with v = 1 - u0 uniform,
 * written with log1p/expm1 for accuracy; accept iff u1^2 <= 1 - a0^2, which
 * is the sqrt(1 - a0^2) Jacobian of the Haar measure.  On acceptance the
 * direction is uniform on S^2: cos(theta) = 2 u2 - 1, phi = 2 pi u3.
 * Returns 1 and fills x on acceptance.
 * Pinned by: a0 histogram against the exact density, acceptance rate
 * against its closed form, isotropy (tests/test_oracle_heatbath.py).
 */
static int creutz_attempt(double k, const double u[4], double x[4])
{
    double a0 = 1.0 + log1p((1.0 - u[0]) * expm1(-2.0 * k)) / k;
    if (!(u[1] * u[1] <= 1.0 - a0 * a0)) return 0;
    double r = sqrt(1.0 - a0 * a0);
    double ct = 2.0 * u[2] - 1.0;
    double st = sqrt(1.0 - ct * ct);
    double phi = TWO_PI * u[3];
    x[0] = a0;
    x[1] = r * st * cos(phi);
    x[2] = r * st * sin(phi);
    x[3] = r * ct;
    return 1;
}

/* Exposed for the sampler tests: n Creutz attempts at fixed k. */
void orc_creutz_samples(double k, uint64_t seed, long n, double* x_out, int* accepted)
{
    for (long t = 0; t < n; t++) {
        double u[4], x[4] = {0, 0, 0, 0};
        draw4(seed, 0, (uint32_t)(t & 0xffffffff), 0, 0, 0, KIND_HB, (uint64_t)(t >> 32), u);
        accepted[t] = creutz_attempt(k, u, x);
        for (int c = 0; c < 4; c++) x_out[4 * t + c] = x[c];
    }
}

/*
 * Heat-bath update of one link U_mu(x) with staple A: V = U A; for each
 * subgroup s in order (0,1), (0,2), (1,2): w from the block of V, xi = |w|,
 * k = 2 beta xi / 3 (the local weight is exp((beta/3) Re Tr(R V))), up to
 * n_hb Creutz attempts; the first accepted X gives R = R(X) R(w/xi), and
 * U <- R U, V <- R V.  A subgroup with no accepted attempt is left as it
 * is.  Finally U is reunitarised.  dec[s] = accepted attempt, 255 if none.
 */
static mat3 hb_link(mat3 Ul, mat3 A, double beta, int n_hb, uint64_t seed, uint32_t lattice_id,
                    long s_lex, int mu, uint64_t sweep, uint8_t* dec)
{
    mat3 V = m_mul(Ul, A);
    for (int s = 0; s < 3; s++) {
        dec[s] = 255;
        double w[4];
        subgroup_w(V, s, w);
        double xi = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        if (xi < 1e-300) continue;
        double k = 2.0 * beta * xi / 3.0;
        for (int att = 0; att < n_hb; att++) {
            double u[4], x[4];
            draw4(seed, lattice_id, (uint32_t)s_lex, mu, s, att, KIND_HB, sweep, u);
            if (creutz_attempt(k, u, x)) {
                double wh[4] = {w[0] / xi, w[1] / xi, w[2] / xi, w[3] / xi};
                mat2 R = m2_mul(quat_to_mat(x), quat_to_mat(wh));
                Ul = embed_left(R, s, Ul);
                V = embed_left(R, s, V);
                dec[s] = (uint8_t)att;
                break;
            }
        }
    }
    return reunit(Ul);
}

/*
 * Overrelaxation of one link: per subgroup R = R(w/xi)^2, the reflection
 * through the maximum of Re Tr(R V) that leaves Re Tr(R V) unchanged; then
 * reunitarise.  Pinned by: the local and total action are preserved; two
 * reflections with a frozen staple in reverse subgroup order give back U.
 */
static mat3 or_link(mat3 Ul, mat3 A)
{
    mat3 V = m_mul(Ul, A);
    for (int s = 0; s < 3; s++) {
        double w[4];
        subgroup_w(V, s, w);
        double xi = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        if (xi < 1e-300) continue;
        double wh[4] = {w[0] / xi, w[1] / xi, w[2] / xi, w[3] / xi};
        mat2 Rw = quat_to_mat(wh);
        mat2 R = m2_mul(Rw, Rw);
        Ul = embed_left(R, s, Ul);
        V = embed_left(R, s, V);
    }
    return reunit(Ul);
}

/* Exposed for tests: the overrelaxation map for a given link and staple, with
 * the subgroups taken in the given order (3 ints). */
void orc_or_link_ordered(const double* Uin, const double* Ain, const int* order, double* Uout)
{
    mat3 Ul, A;
    memcpy(&Ul, Uin, sizeof Ul);
    memcpy(&A, Ain, sizeof A);
    mat3 V = m_mul(Ul, A);
    for (int t = 0; t < 3; t++) {
        int s = order[t];
        double w[4];
        subgroup_w(V, s, w);
        double xi = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        if (xi < 1e-300) continue;
        double wh[4] = {w[0] / xi, w[1] / xi, w[2] / xi, w[3] / xi};
        mat2 Rw = quat_to_mat(wh);
        mat2 R = m2_mul(Rw, Rw);
        Ul = embed_left(R, s, Ul);
        V = embed_left(R, s, V);
    }
    memcpy(Uout, &Ul, sizeof Ul);
}

/*
 * One heat-bath sweep on the checkerboard schedule: for mu = 0..3, for
 * parity = 0, 1, update every link U_mu(x) with x of that parity.  Links of
 * one (mu, parity) subset share no plaquette, so their order is irrelevant.
 * dec (optional) receives dec[(site*4 + mu)*3 + subgroup].
 */
void orc_heatbath_sweep(double* U, const int* dims, double beta, uint64_t seed, uint32_t lattice_id,
                        uint64_t sweep, int n_hb, uint8_t* dec)
{
    lat_t g = make_lat(dims);
    for (int mu = 0; mu < 4; mu++)
        for (int par = 0; par < 2; par++) {
#pragma omp parallel for schedule(static)
            for (long s = 0; s < g.V; s++) {
                if (parity_of(&g, s) != par) continue;
                uint8_t d[3];
                mat3 A = staple(&g, U, s, mu);
                mat3 Un = hb_link(getU(U, s, mu), A, beta, n_hb, seed, lattice_id, s, mu, sweep, d);
                setU(U, s, mu, Un);
                if (dec) memcpy(dec + ((size_t)s * 4 + mu) * 3, d, 3);
            }
        }
}

/* One (mu, parity) subset only; same semantics as one step of the sweep. */
void orc_heatbath_subsweep(double* U, const int* dims, double beta, uint64_t seed, uint32_t lattice_id,
                           uint64_t sweep, int n_hb, int mu, int par, uint8_t* dec)
{
    lat_t g = make_lat(dims);
    mat3* Unew = malloc(sizeof(mat3) * g.V);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++) {
        if (parity_of(&g, s) != par) continue;
        uint8_t d[3];
        mat3 A = staple(&g, U, s, mu);
        Unew[s] = hb_link(getU(U, s, mu), A, beta, n_hb, seed, lattice_id, s, mu, sweep, d);
        if (dec) memcpy(dec + ((size_t)s * 4 + mu) * 3, d, 3);
    }
    for (long s = 0; s < g.V; s++)
        if (parity_of(&g, s) == par) setU(U, s, mu, Unew[s]);
    free(Unew);
}

/* The heat-bath result for a single link, without modifying U. */
void orc_heatbath_one_link(const double* U, const int* dims, double beta, uint64_t seed, uint32_t lattice_id,
                           uint64_t sweep, int n_hb, long s, int mu, double* Uout, uint8_t* dec)
{
    lat_t g = make_lat(dims);
    mat3 A = staple(&g, U, s, mu);
    mat3 Un = hb_link(getU(U, s, mu), A, beta, n_hb, seed, lattice_id, s, mu, sweep, dec);
    memcpy(Uout, &Un, sizeof Un);
}

/* The heat-bath result for a link U_in with staple A_in (both 3x3, row-major
 * complex), as the link of direction mu at lexicographic site s_lex would get
 * it in the given sweep: the same map as orc_heatbath_one_link with the staple
 * supplied by the caller, for links of lattices too large to hold here. */
void orc_heatbath_link_staple(const double* Uin, const double* Ain, double beta, uint64_t seed, uint32_t lattice_id,
                              uint64_t sweep, int n_hb, long s_lex, int mu, double* Uout, uint8_t* dec)
{
    mat3 Ul, A;
    memcpy(&Ul, Uin, sizeof Ul);
    memcpy(&A, Ain, sizeof A);
    mat3 Un = hb_link(Ul, A, beta, n_hb, seed, lattice_id, s_lex, mu, sweep, dec);
    memcpy(Uout, &Un, sizeof Un);
}

/* One overrelaxation sweep on the same checkerboard schedule (no RNG). */
void orc_overrelax_sweep(double* U, const int* dims)
{
    lat_t g = make_lat(dims);
    for (int mu = 0; mu < 4; mu++)
        for (int par = 0; par < 2; par++) {
#pragma omp parallel for schedule(static)
            for (long s = 0; s < g.V; s++) {
                if (parity_of(&g, s) != par) continue;
                mat3 A = staple(&g, U, s, mu);
                setU(U, s, mu, or_link(getU(U, s, mu), A));
            }
        }
}

/*
 * The same (mu, parity) updates restricted to the sites with lexicographic
 * index in [s_lo, s_hi) (a slab of x3 planes when the bounds are multiples of
 * L0 L1 L2); used to time bounded samples of a sweep.  kind 0 = heat bath,
 * 1 = overrelaxation.
 */
void orc_subsweep_range(double* U, const int* dims, int kind, double beta, uint64_t seed, uint32_t lattice_id,
                        uint64_t sweep, int n_hb, int mu, int par, long s_lo, long s_hi)
{
    lat_t g = make_lat(dims);
#pragma omp parallel for schedule(static)
    for (long s = s_lo; s < s_hi; s++) {
        if (parity_of(&g, s) != par) continue;
        uint8_t d[3];
        mat3 A = staple(&g, U, s, mu);
        mat3 Un = kind == 0 ? hb_link(getU(U, s, mu), A, beta, n_hb, seed, lattice_id, s, mu, sweep, d)
                            : or_link(getU(U, s, mu), A);
        setU(U, s, mu, Un);
    }
}

/* One (mu, parity) subset of the overrelaxation sweep. */
void orc_overrelax_subsweep(double* U, const int* dims, int mu, int par)
{
    lat_t g = make_lat(dims);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++) {
        if (parity_of(&g, s) != par) continue;
        mat3 A = staple(&g, U, s, mu);
        setU(U, s, mu, or_link(getU(U, s, mu), A));
    }
}

/* The overrelaxation result for a single link, without modifying U. */
void orc_overrelax_one_link(const double* U, const int* dims, long s, int mu, double* Uout)
{
    lat_t g = make_lat(dims);
    mat3 Un = or_link(getU(U, s, mu), staple(&g, U, s, mu));
    memcpy(Uout, &Un, sizeof Un);
}

/*
 * n_sweeps x (1 heat-bath sweep + n_or overrelaxation sweeps); the heat-bath
 * sweep index is sweep0 + i.  plaq_out (optional, n_sweeps) receives the
 * average plaquette after each compound sweep.
 */
void orc_update_chain(double* U, const int* dims, double beta, uint64_t seed, uint32_t lattice_id,
                      uint64_t sweep0, int n_sweeps, int n_hb, int n_or, double* plaq_out)
{
    for (int i = 0; i < n_sweeps; i++) {
        orc_heatbath_sweep(U, dims, beta, seed, lattice_id, sweep0 + (uint64_t)i, n_hb, NULL);
        for (int j = 0; j < n_or; j++) orc_overrelax_sweep(U, dims);
        if (plaq_out) plaq_out[i] = orc_plaquette(U, dims);
    }
}

/* ------------------------------------------------------------------------ */
/* su(3) algebra: X_a = i lambda_a / 2 with the Gell-Mann matrices.          */
/* ------------------------------------------------------------------------ */
static mat3 gell_mann(int a)
{
    mat3 l = m_zero();
    switch (a) {
    case 0: l.e[0][1] = 1; l.e[1][0] = 1; break;
    case 1: l.e[0][1] = -I; l.e[1][0] = I; break;
    case 2: l.e[0][0] = 1; l.e[1][1] = -1; break;
    case 3: l.e[0][2] = 1; l.e[2][0] = 1; break;
    case 4: l.e[0][2] = -I; l.e[2][0] = I; break;
    case 5: l.e[1][2] = 1; l.e[2][1] = 1; break;
    case 6: l.e[1][2] = -I; l.e[2][1] = I; break;
    case 7: {
        double s = 1.0 / sqrt(3.0);
        l.e[0][0] = s; l.e[1][1] = s; l.e[2][2] = -2.0 * s;
        break;
    }
    }
    return l;
}

static mat3 gen_X(int a) { return m_scale(gell_mann(a), 0.5 * I); }

/* Sum_a p_a X_a */
static mat3 alg_to_mat(const double* p)
{
    mat3 r = m_zero();
    for (int a = 0; a < 8; a++) r = m_add(r, m_scale(gen_X(a), p[a]));
    return r;
}

/* coefficients of an anti-hermitian traceless Y:  p_a = -2 Tr(X_a Y) */
static void mat_to_alg(mat3 Y, double* p)
{
    for (int a = 0; a < 8; a++) p[a] = -2.0 * creal(m_trace(m_mul(gen_X(a), Y)));
}

/* Traceless anti-hermitian part TA(M) = (M - M^+)/2 - Tr((M - M^+)/2)/3 */
static mat3 traceless_antiherm(mat3 M)
{
    mat3 ah = m_scale(m_sub(M, m_dag(M)), 0.5);
    cplx t = m_trace(ah) / 3.0;
    for (int i = 0; i < 3; i++) ah.e[i][i] -= t;
    return ah;
}

/*
 * exp(X) of a 3x3 matrix from its series definition, sum_n X^n/n!, evaluated
 * on X/2^m (Frobenius norm <= 1/2, 30 terms) and squared m times.
 * Pinned by: scipy.linalg.expm; exp(-X) exp(X) = 1; det = exp(Tr X).
 */
static mat3 expm3(mat3 X)
{
    double nrm = m_frob(X);
    int m = 0;
    while (nrm > 0.5) { nrm *= 0.5; m++; }
    mat3 Y = m_scale(X, ldexp(1.0, -m));
    mat3 T = m_unit(), term = m_unit();
    for (int n = 1; n <= 30; n++) {
        term = m_scale(m_mul(term, Y), 1.0 / n);
        T = m_add(T, term);
    }
    for (int i = 0; i < m; i++) T = m_mul(T, T);
    return T;
}

void orc_expm(const double* X, double* out)
{
    mat3 x, r;
    memcpy(&x, X, sizeof x);
    r = expm3(x);
    memcpy(out, &r, sizeof r);
}

void orc_alg_to_mat(const double* p, double* out)
{
    mat3 r = alg_to_mat(p);
    memcpy(out, &r, sizeof r);
}

void orc_mat_to_alg(const double* M, double* p)
{
    mat3 m;
    memcpy(&m, M, sizeof m);
    mat_to_alg(m, p);
}

/* ------------------------------------------------------------------------ */
/* HMC (Sec. IV.D; PQP leapfrog with unit-length trajectories).              */
/* ------------------------------------------------------------------------ */

/*
 * Gauge force in algebra coefficients, F(x,mu) = -(beta/6) TA(U_mu(x) A_mu(x)):
 * the EOM dP/dt for the Hamiltonian H = sum p_a^2/2 + S with dU/dt = P U.
 * Pinned by: central finite differences of S along each generator;
 * zero on the unit gauge; gauge covariance.
 */
void orc_force(const double* U, const int* dims, double beta, double* F)
{
    lat_t g = make_lat(dims);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++)
        for (int mu = 0; mu < 4; mu++) {
            mat3 M = m_mul(getU(U, s, mu), staple(&g, U, s, mu));
            mat3 Fm = m_scale(traceless_antiherm(M), -beta / 6.0);
            mat_to_alg(Fm, F + ((size_t)s * 4 + mu) * 8);
        }
}

/* Gaussian momenta: p_a ~ N(0,1), 8 per link from two draws (Box-Muller). */
void orc_mom_refresh(double* P, const int* dims, uint64_t seed, uint32_t lattice_id, uint64_t traj)
{
    lat_t g = make_lat(dims);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++)
        for (int mu = 0; mu < 4; mu++) {
            double* p = P + ((size_t)s * 4 + mu) * 8;
            for (int call = 0; call < 2; call++) {
                double u[4];
                draw4(seed, lattice_id, (uint32_t)s, mu, 0, call, KIND_MOM, traj, u);
                box_muller(u[0], u[1], &p[4 * call + 0], &p[4 * call + 1]);
                box_muller(u[2], u[3], &p[4 * call + 2], &p[4 * call + 3]);
            }
        }
}

double orc_kinetic(const double* P, const int* dims)
{
    lat_t g = make_lat(dims);
    double acc = 0;
    for (size_t i = 0; i < (size_t)g.V * 32; i++) acc += 0.5 * P[i] * P[i];
    return acc;
}

/* U <- exp(eps P) U on every link */
void orc_update_links(double* U, const double* P, const int* dims, double eps)
{
    lat_t g = make_lat(dims);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++)
        for (int mu = 0; mu < 4; mu++) {
            mat3 Pm = alg_to_mat(P + ((size_t)s * 4 + mu) * 8);
            setU(U, s, mu, m_mul(expm3(m_scale(Pm, eps)), getU(U, s, mu)));
        }
}

/* P <- P + eps F(U) */
static void update_mom(double* P, const double* U, const int* dims, double beta, double eps, double* Fbuf)
{
    lat_t g = make_lat(dims);
    orc_force(U, dims, beta, Fbuf);
    for (size_t i = 0; i < (size_t)g.V * 32; i++) P[i] += eps * Fbuf[i];
}

/*
 * Leapfrog integration of n_steps steps of size eps = tau/n_steps in the PQP
 * order: P(eps/2) [Q(eps) P(eps)]^(n-1) Q(eps) P(eps/2), where the inner
 * pairs of half-steps are merged into one full P step.
 */
void orc_leapfrog(double* U, double* P, const int* dims, double beta, double tau, int n_steps)
{
    lat_t g = make_lat(dims);
    double eps = tau / n_steps;
    double* F = malloc(sizeof(double) * g.V * 32);
    update_mom(P, U, dims, beta, 0.5 * eps, F);
    for (int st = 0; st < n_steps; st++) {
        orc_update_links(U, P, dims, eps);
        update_mom(P, U, dims, beta, (st == n_steps - 1) ? 0.5 * eps : eps, F);
    }
    free(F);
}

/*
 * One HMC trajectory: momenta from the MOM stream of trajectory traj,
 * H0 = T + S, leapfrog, H1, dH = H1 - H0; accept iff u < exp(-dH) with u
 * the first uniform of the ACCEPT draw of trajectory traj (site 0, mu 0);
 * accept_reject = 0 always accepts (warm-up).  A rejection restores U.
 * Pinned by: reversibility, dH ~ eps^2, <exp(-dH)> = 1.
 */
void orc_hmc_trajectory(double* U, double* P, const int* dims, double beta, double tau, int n_steps,
                        uint64_t seed, uint32_t lattice_id, uint64_t traj, int accept_reject,
                        double* dH_out, int* accepted_out)
{
    lat_t g = make_lat(dims);
    size_t nU = (size_t)g.V * 72;
    double* U0 = malloc(sizeof(double) * nU);
    memcpy(U0, U, sizeof(double) * nU);
    orc_mom_refresh(P, dims, seed, lattice_id, traj);
    double H0 = orc_kinetic(P, dims) + orc_action(U, dims, beta);
    orc_leapfrog(U, P, dims, beta, tau, n_steps);
    double H1 = orc_kinetic(P, dims) + orc_action(U, dims, beta);
    double dH = H1 - H0;
    double u[4];
    draw4(seed, lattice_id, 0, 0, 0, 0, KIND_ACCEPT, traj, u);
    int acc = accept_reject ? (u[0] < exp(-dH)) : 1;
    if (!acc) memcpy(U, U0, sizeof(double) * nU);
    free(U0);
    *dH_out = dH;
    *accepted_out = acc;
}

/* ------------------------------------------------------------------------ */
/* Projection onto SU(3) (Eq. APE: P_SU(Nc)).                                */
/* ------------------------------------------------------------------------ */

/*
 * P_SU(3)(M): start from the Gram-Schmidt SU(3) matrix W of M, then n_pass
 * passes over the subgroups (0,1), (0,2), (1,2), each replacing W by
 * R W with R the SU(2) element maximising Re Tr(R W M^+) (R = R(w/xi),
 * w from the block of W M^+).  Re Tr(W M^+) never decreases.
 * Pinned by: P(M) = M on SU(3); P(H U) -> U for positive hermitian H as
 * the pass count grows; P(s U) = U for s > 0.
 */
static mat3 su3_project(mat3 M, int n_pass)
{
    mat3 W = reunit(M);
    mat3 Md = m_dag(M);
    for (int pass = 0; pass < n_pass; pass++)
        for (int s = 0; s < 3; s++) {
            double w[4];
            subgroup_w(m_mul(W, Md), s, w);
            double xi = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
            if (xi < 1e-300) continue;
            double wh[4] = {w[0] / xi, w[1] / xi, w[2] / xi, w[3] / xi};
            W = embed_left(quat_to_mat(wh), s, W);
        }
    return W;
}

void orc_su3_project(const double* M, int n_pass, double* out)
{
    mat3 m, r;
    memcpy(&m, M, sizeof m);
    r = su3_project(m, n_pass);
    memcpy(out, &r, sizeof r);
}

void orc_reunit(const double* M, double* out)
{
    mat3 m, r;
    memcpy(&m, M, sizeof m);
    r = reunit(m);
    memcpy(out, &r, sizeof r);
}

/* ------------------------------------------------------------------------ */
/* Restriction and prolongation (Sec. III, Eqs. restriction, prolongation,   */
/* smoothing, APE).                                                          */
/* ------------------------------------------------------------------------ */

/* chi_mu(n) = number of odd coordinates of n other than n_mu */
static int chi_mu(const int x[4], int mu)
{
    int c = 0;
    for (int nu = 0; nu < 4; nu++)
        if (nu != mu) c += x[nu] & 1;
    return c;
}

/* chi_munu(n) = number of odd coordinates of n other than n_mu, n_nu */
static int chi_munu(const int x[4], int mu, int nu)
{
    int c = 0;
    for (int r = 0; r < 4; r++)
        if (r != mu && r != nu) c += x[r] & 1;
    return c;
}

/*
 * Restriction: U^c_mu(n/2) = U^f_mu(n) U^f_mu(n + e_mu) for chi(n) = 0.
 * Fine extents are twice the coarse ones.
 */
void orc_restrict(const double* Uf, const int* dims_f, double* Uc)
{
    lat_t gf = make_lat(dims_f);
    int dc[4] = {dims_f[0] / 2, dims_f[1] / 2, dims_f[2] / 2, dims_f[3] / 2};
    lat_t gc = make_lat(dc);
    for (long sc = 0; sc < gc.V; sc++) {
        int xc[4], xf[4];
        coords_of(&gc, sc, xc);
        for (int mu = 0; mu < 4; mu++) xf[mu] = 2 * xc[mu];
        long sf = site_of(&gf, xf);
        for (int mu = 0; mu < 4; mu++)
            setU(Uc, sc, mu, m_mul(getU(Uf, sf, mu), getU(Uf, hop(&gf, sf, mu, +1), mu)));
    }
}

/*
 * Transfer (Eq. prolongation): for n with chi(n) = 0,
 * U^f_mu(n) = U^c_mu(n/2) and U^f_mu(n + e_mu) = 1; every other fine bond
 * starts at 1.
 */
void orc_transfer(const double* Uc, const int* dims_c, double* Uf)
{
    int df[4] = {2 * dims_c[0], 2 * dims_c[1], 2 * dims_c[2], 2 * dims_c[3]};
    lat_t gf = make_lat(df), gc = make_lat(dims_c);
    for (long sf = 0; sf < gf.V; sf++)
        for (int mu = 0; mu < 4; mu++) setU(Uf, sf, mu, m_unit());
    for (long sc = 0; sc < gc.V; sc++) {
        int xc[4], xf[4];
        coords_of(&gc, sc, xc);
        for (int mu = 0; mu < 4; mu++) xf[mu] = 2 * xc[mu];
        long sf = site_of(&gf, xf);
        for (int mu = 0; mu < 4; mu++) setU(Uf, sf, mu, getU(Uc, sc, mu));
    }
}

/*
 * Partial action S_d / beta = sum_n sum_{mu<nu} delta_{d, chi_munu(n)} [1 - W_munu(n)]
 * (Eq. smoothing, without the overall beta).
 */
double orc_partial_action(const double* U, const int* dims, int d)
{
    lat_t g = make_lat(dims);
    double* part = malloc(sizeof(double) * g.V);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++) {
        int x[4];
        coords_of(&g, s, x);
        double acc = 0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++)
                if (chi_munu(x, mu, nu) == d) acc += 1.0 - creal(m_trace(plaq_mat(&g, U, s, mu, nu))) / 3.0;
        part[s] = acc;
    }
    double acc = 0;
    for (long s = 0; s < g.V; s++) acc += part[s];
    free(part);
    return acc;
}

/*
 * One APE step of stage d (Eq. APE), all active bonds at once (Jacobi):
 * active bonds have chi_mu(n) = d + 1, and the staple directions nu are
 * those with delta_{d, chi_munu(n)} = 1, i.e. n_nu odd.
 * T+_munu(n) = U_nu(n) U_mu(n+nu) U_nu(n+mu)^+
 * T-_munu(n) = U_nu(n-nu)^+ U_mu(n-nu) U_nu(n-nu+mu)
 * (the printed T- carries a dagger on its last factor, which is not gauge
 * covariant; the backward staple above is).  Pinned by: a pure-gauge field is
 * a fixed point of every stage; the step commutes with local gauge
 * transforms; on abelian links diag(e^{it}, e^{-it}, 1) it is U(1) APE
 * smearing of t (tests/test_oracle_prolong.py).
 */
static void ape_step(double* U, double* Unew, const lat_t* g, int d, double c, int n_pass)
{
    size_t nU = (size_t)g->V * 72;
    memcpy(Unew, U, sizeof(double) * nU);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g->V; s++) {
        int x[4];
        coords_of(g, s, x);
        for (int mu = 0; mu < 4; mu++) {
            if (chi_mu(x, mu) != d + 1) continue;
            mat3 M = getU(U, s, mu);
            for (int nu = 0; nu < 4; nu++) {
                if (nu == mu || chi_munu(x, mu, nu) != d) continue;
                long xpn = hop(g, s, nu, +1), xpm = hop(g, s, mu, +1), xmn = hop(g, s, nu, -1);
                long xmn_pm = hop2(g, s, nu, -1, mu, +1);
                mat3 tp = m_mul(m_mul(getU(U, s, nu), getU(U, xpn, mu)), m_dag(getU(U, xpm, nu)));
                mat3 tm = m_mul(m_mul(m_dag(getU(U, xmn, nu)), getU(U, xmn, mu)), getU(U, xmn_pm, nu));
                M = m_add(M, m_scale(m_add(tp, tm), c));
            }
            setU(Unew, s, mu, su3_project(M, n_pass));
        }
    }
    memcpy(U, Unew, sizeof(double) * nU);
}

/* One APE step of stage d on the field U in place (exposed for the pins). */
void orc_ape_step(double* U, const int* dims, int d, double c, int n_pass)
{
    lat_t g = make_lat(dims);
    double* tmp = malloc(sizeof(double) * g.V * 72);
    ape_step(U, tmp, &g, d, c, n_pass);
    free(tmp);
}

/*
 * Prolongation = transfer, then interpolation stages d = 0, 1, 2 in order;
 * each stage repeats APE steps until the relative change of S_d between
 * consecutive steps is <= rel_tol, or max_iter steps (rel_tol <= 0: exactly
 * max_iter steps).  iters_out[d] = steps taken; sd_out (optional, 3) = final
 * S_d / beta.
 */
void orc_prolongate(const double* Uc, const int* dims_c, double* Uf, double c, double rel_tol,
                    int max_iter, int n_pass, int* iters_out, double* sd_out)
{
    int df[4] = {2 * dims_c[0], 2 * dims_c[1], 2 * dims_c[2], 2 * dims_c[3]};
    lat_t gf = make_lat(df);
    orc_transfer(Uc, dims_c, Uf);
    double* tmp = malloc(sizeof(double) * gf.V * 72);
    for (int d = 0; d <= 2; d++) {
        double prev = orc_partial_action(Uf, df, d);
        int it = 0;
        double cur = prev;
        while (it < max_iter) {
            ape_step(Uf, tmp, &gf, d, c, n_pass);
            it++;
            cur = orc_partial_action(Uf, df, d);
            if (rel_tol > 0 && fabs(cur - prev) <= rel_tol * fabs(prev)) break;
            prev = cur;
        }
        iters_out[d] = it;
        if (sd_out) sd_out[d] = cur;
    }
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Wilson loops and the rethermalisation diagnostics (Sec. III: Wilson      */
/* lines, m x n loops, partial plaquettes, displaced 2x2 loops; Sec. IV.C:  */
/* smoothness s_p and admissibility).                                        */
/* ------------------------------------------------------------------------ */

/* Wilson line L^m_mu(x) = U_mu(x) U_mu(x+mu) ... U_mu(x+(m-1)mu) */
static mat3 wilson_line(const lat_t* g, const double* U, long s, int mu, int m)
{
    mat3 L = m_unit();
    for (int k = 0; k < m; k++) {
        L = m_mul(L, getU(U, s, mu));
        s = hop(g, s, mu, +1);
    }
    return L;
}

/* W^{m x n}_munu(x) = (1/3) Re Tr L^m_mu(x) L^n_nu(x+m mu) L^m_mu(x+n nu)^+ L^n_nu(x)^+ */
static double loop_mn(const lat_t* g, const double* U, long s, int mu, int nu, int m, int n)
{
    long xm = s, xn = s;
    for (int k = 0; k < m; k++) xm = hop(g, xm, mu, +1);
    for (int k = 0; k < n; k++) xn = hop(g, xn, nu, +1);
    mat3 a = m_mul(wilson_line(g, U, s, mu, m), wilson_line(g, U, xm, nu, n));
    mat3 b = m_mul(wilson_line(g, U, s, nu, n), wilson_line(g, U, xn, mu, m));
    return creal(m_trace(m_mul(a, m_dag(b)))) / 3.0;
}

/* Space-time average of the m x n loops over all x and mu < nu, normalised by N_2 = 6 V. */
double orc_wilson_loop(const double* U, const int* dims, int m, int n)
{
    lat_t g = make_lat(dims);
    double* part = malloc(sizeof(double) * g.V);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++) {
        double acc = 0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) acc += loop_mn(&g, U, s, mu, nu, m, n);
        part[s] = acc;
    }
    double acc = 0;
    for (long s = 0; s < g.V; s++) acc += part[s];
    free(part);
    return acc / (6.0 * (double)g.V);
}

static double binom(int n, int k)
{
    double r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

/*
 * out[0..2]: partial plaquettes W^{1x1}_d = (1/N^{1x1}_d) sum over plaquettes
 *            with chi_munu(n) = d of W^{1x1}_munu(n),
 *            N^{1x1}_d = 2 (D-d)(D-d-1) C(D,d) N_0 / 2^D;
 * out[3..7]: displaced loops W^{2x2}_d = (1/N^{2x2}_d) sum over (n, mu<nu)
 *            with chi(n) = d of W^{2x2}_munu(n), N^{2x2}_d = C(D,2) C(D,d) N_0 / 2^D;
 * out[8]   : h = max_p s_p, s_p = N_c [1 - W^{1x1}_p].
 * Defined for lattices with even extents; the d classes refer to the coarse
 * lattice of the even sites.
 */
void orc_partial_loops(const double* U, const int* dims, double* out)
{
    lat_t g = make_lat(dims);
    const int D = 4;
    double* p1 = calloc((size_t)g.V * 3, sizeof(double));
    double* p2 = calloc((size_t)g.V * 5, sizeof(double));
    double* hx = calloc((size_t)g.V, sizeof(double));
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++) {
        int x[4];
        coords_of(&g, s, x);
        int chi = 0;
        for (int r = 0; r < 4; r++) chi += x[r] & 1;
        double hmax = 0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                double w1 = loop_mn(&g, U, s, mu, nu, 1, 1);
                p1[(size_t)s * 3 + chi_munu(x, mu, nu)] += w1;
                p2[(size_t)s * 5 + chi] += loop_mn(&g, U, s, mu, nu, 2, 2);
                double sp = 3.0 * (1.0 - w1);
                if (sp > hmax) hmax = sp;
            }
        hx[s] = hmax;
    }
    double a1[3] = {0, 0, 0}, a2[5] = {0, 0, 0, 0, 0}, h = 0;
    for (long s = 0; s < g.V; s++) {
        for (int d = 0; d < 3; d++) a1[d] += p1[(size_t)s * 3 + d];
        for (int d = 0; d < 5; d++) a2[d] += p2[(size_t)s * 5 + d];
        if (hx[s] > h) h = hx[s];
    }
    for (int d = 0; d < 3; d++) out[d] = a1[d] / (2.0 * (D - d) * (D - d - 1) * binom(D, d) * (double)g.V / 16.0);
    for (int d = 0; d < 5; d++) out[3 + d] = a2[d] / (binom(D, 2) * binom(D, d) * (double)g.V / 16.0);
    out[8] = h;
    free(p1); free(p2); free(hx);
}

/* ------------------------------------------------------------------------ */
/* Wilson flow (Sec. IV.B, fixed step, Luscher's third-order Runge-Kutta)    */
/* and clover observables E(t), Q(t).                                        */
/* ------------------------------------------------------------------------ */

/*
 * Flow generator Z(W)(x,mu) = -TA(W_mu(x) A_mu(x)): minus the Lie derivative
 * of the Wilson action times g0^2 = 6/beta, i.e. the HMC force at beta = 6.
 * Pinned by: a small abelian plane wave decays as exp(-t p^2) with the
 * lattice momentum p^2 = sum 4 sin^2(p_nu/2).
 */
static void flow_generator(const lat_t* g, const double* W, mat3* Z, double scale)
{
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g->V; s++)
        for (int mu = 0; mu < 4; mu++) {
            mat3 M = m_mul(getU(W, s, mu), staple(g, W, s, mu));
            Z[s * 4 + mu] = m_scale(traceless_antiherm(M), -scale);
        }
}

/* W <- exp(X) W on every link */
static void exp_update(const lat_t* g, double* W, const mat3* X)
{
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g->V; s++)
        for (int mu = 0; mu < 4; mu++) setU(W, s, mu, m_mul(expm3(X[s * 4 + mu]), getU(W, s, mu)));
}

/*
 * One step of size eps:
 *   W1 = exp(Z0/4) W0
 *   W2 = exp(8/9 Z1 - 17/36 Z0) W1
 *   W3 = exp(3/4 Z2 - 8/9 Z1 + 17/36 Z0) W2,   Z_i = eps Z(W_i).
 */
void orc_flow_step(double* W, const int* dims, double eps)
{
    lat_t g = make_lat(dims);
    size_t n = (size_t)g.V * 4;
    mat3* Z0 = malloc(sizeof(mat3) * n);
    mat3* Z1 = malloc(sizeof(mat3) * n);
    mat3* Z2 = malloc(sizeof(mat3) * n);
    mat3* X = malloc(sizeof(mat3) * n);
    flow_generator(&g, W, Z0, eps);
    for (size_t i = 0; i < n; i++) X[i] = m_scale(Z0[i], 0.25);
    exp_update(&g, W, X);
    flow_generator(&g, W, Z1, eps);
    for (size_t i = 0; i < n; i++) X[i] = m_sub(m_scale(Z1[i], 8.0 / 9.0), m_scale(Z0[i], 17.0 / 36.0));
    exp_update(&g, W, X);
    flow_generator(&g, W, Z2, eps);
    for (size_t i = 0; i < n; i++)
        X[i] = m_add(m_sub(m_scale(Z2[i], 0.75), m_scale(Z1[i], 8.0 / 9.0)), m_scale(Z0[i], 17.0 / 36.0));
    exp_update(&g, W, X);
    free(Z0); free(Z1); free(Z2); free(X);
}

/*
 * Clover field strength at x in the (mu,nu) plane: Q_munu = the four
 * plaquette leaves around x, all starting and ending at x, counterclockwise;
 * G_munu = (Q_munu - Q_munu^+)/8 made traceless.
 */
static mat3 clover_G(const lat_t* g, const double* U, long s, int mu, int nu)
{
    long xpm = hop(g, s, mu, +1), xpn = hop(g, s, nu, +1);
    long xmm = hop(g, s, mu, -1), xmn = hop(g, s, nu, -1);
    long xmm_pn = hop2(g, s, mu, -1, nu, +1);
    long xmm_mn = hop2(g, s, mu, -1, nu, -1);
    long xpm_mn = hop2(g, s, mu, +1, nu, -1);
    mat3 l1 = m_mul(m_mul(getU(U, s, mu), getU(U, xpm, nu)), m_mul(m_dag(getU(U, xpn, mu)), m_dag(getU(U, s, nu))));
    mat3 l2 = m_mul(m_mul(getU(U, s, nu), m_dag(getU(U, xmm_pn, mu))),
                    m_mul(m_dag(getU(U, xmm, nu)), getU(U, xmm, mu)));
    mat3 l3 = m_mul(m_mul(m_dag(getU(U, xmm, mu)), m_dag(getU(U, xmm_mn, nu))),
                    m_mul(getU(U, xmm_mn, mu), getU(U, xmn, nu)));
    mat3 l4 = m_mul(m_mul(m_dag(getU(U, xmn, nu)), getU(U, xmn, mu)), m_mul(getU(U, xpm_mn, nu), m_dag(getU(U, s, mu))));
    mat3 Qm = m_add(m_add(l1, l2), m_add(l3, l4));
    mat3 G = m_scale(m_sub(Qm, m_dag(Qm)), 0.125);
    cplx t = m_trace(G) / 3.0;
    for (int i = 0; i < 3; i++) G.e[i][i] -= t;
    return G;
}

/*
 * Clover energy density and charge:
 *   E = (1/V) sum_x -1/2 sum_{mu,nu} Tr(G_munu G_munu)
 *   Q = -1/(32 pi^2) sum_x eps_{munurhosigma} Tr(G_munu G_rhosigma)
 *     = -1/(4 pi^2) sum_x [Tr(G01 G23) - Tr(G02 G13) + Tr(G03 G12)]
 * Pinned by: closed forms for a constant abelian flux configuration;
 * gauge invariance.
 */
void orc_clover_EQ(const double* U, const int* dims, double* E_out, double* Q_out)
{
    lat_t g = make_lat(dims);
    double* pe = malloc(sizeof(double) * g.V);
    double* pq = malloc(sizeof(double) * g.V);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++) {
        mat3 G[4][4];
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) G[mu][nu] = clover_G(&g, U, s, mu, nu);
        double e = 0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) e -= creal(m_trace(m_mul(G[mu][nu], G[mu][nu])));
        pe[s] = e; /* -1/2 sum over ordered pairs = - sum over mu<nu */
        double q = creal(m_trace(m_mul(G[0][1], G[2][3]))) - creal(m_trace(m_mul(G[0][2], G[1][3]))) +
                   creal(m_trace(m_mul(G[0][3], G[1][2])));
        pq[s] = -q / (4.0 * M_PI * M_PI);
    }
    double es = 0, qs = 0;
    for (long s = 0; s < g.V; s++) { es += pe[s]; qs += pq[s]; }
    free(pe); free(pq);
    *E_out = es / (double)g.V;
    *Q_out = qs;
}

/*
 * Three-loop improved topological charge (Sec. IV.C, the gluonic operator of
 * de Forcrand, Garcia Perez and Stamatescu, Nucl. Phys. B 499 (1997) 409).
 * q_m(x) is the clover charge density built from the four m x m leaves around
 * x in every plane; an m x m clover on spacing a is the 1 x 1 clover on
 * spacing m a, so for a smooth field q_m(x) = (m a)^4 [q + (m a)^2 X + (m a)^4 Y
 * + O(a^6)].  The combination sum_m c_m q_m / m^4 over m = 1, 2, 3 with
 *   sum c_m = 1,  sum c_m m^2 = 0,  sum c_m m^4 = 0
 * removes the O(a^2) and O(a^4) terms at tree level: c = (3/2, -3/5, 1/10).
 * Pinned by: the exact m x m charges of a constant abelian flux, the L^-8
 * approach of the improved charge to the integer on it, the O(a^6) accuracy
 * of the improved density on a smooth field, gauge invariance
 * (tests/test_oracle_topo.py).
 */
static const double IMPROVED_C[3] = {1.5, -0.6, 0.1};

/* Product of the links along a path of n unit steps from site s: a step along
 * +dir multiplies by U_dir(y), a step along -dir by U_dir(y - dir)^+. */
static mat3 path_product(const lat_t* g, const double* U, long s, const int* dir, const int* sgn, int n)
{
    mat3 P = m_unit();
    long y = s;
    for (int k = 0; k < n; k++) {
        if (sgn[k] > 0) {
            P = m_mul(P, getU(U, y, dir[k]));
            y = hop(g, y, dir[k], +1);
        } else {
            y = hop(g, y, dir[k], -1);
            P = m_mul(P, m_dag(getU(U, y, dir[k])));
        }
    }
    return P;
}

/* Clover field strength from the four m x m leaves around x in the (mu,nu)
 * plane, each starting and ending at x, counterclockwise (the m = 1 leaves of
 * clover_G): G = traceless part of (Q - Q^+)/8, about m^2 a^2 F_munu. */
static mat3 clover_G_m(const lat_t* g, const double* U, long s, int mu, int nu, int m)
{
    const int a[4] = {mu, nu, mu, nu}, sa[4] = {+1, +1, -1, -1};
    const int b[4] = {nu, mu, nu, mu}, sb[4] = {+1, -1, -1, +1};
    mat3 Q = m_scale(m_unit(), 0.0);
    for (int l = 0; l < 4; l++) {
        int dir[12], sgn[12];
        for (int k = 0; k < m; k++) {
            dir[k] = a[l]; sgn[k] = sa[l];
            dir[m + k] = b[l]; sgn[m + k] = sb[l];
            dir[2 * m + k] = a[l]; sgn[2 * m + k] = -sa[l];
            dir[3 * m + k] = b[l]; sgn[3 * m + k] = -sb[l];
        }
        Q = m_add(Q, path_product(g, U, s, dir, sgn, 4 * m));
    }
    mat3 G = m_scale(m_sub(Q, m_dag(Q)), 0.125);
    cplx t = m_trace(G) / 3.0;
    for (int i = 0; i < 3; i++) G.e[i][i] -= t;
    return G;
}

/* q_m(x) = -1/(4 pi^2) [Tr(G01 G23) - Tr(G02 G13) + Tr(G03 G12)] from m x m leaves */
static double clover_q_m(const lat_t* g, const double* U, long s, int m)
{
    mat3 G[4][4];
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++) G[mu][nu] = clover_G_m(g, U, s, mu, nu, m);
    double q = creal(m_trace(m_mul(G[0][1], G[2][3]))) - creal(m_trace(m_mul(G[0][2], G[1][3]))) +
               creal(m_trace(m_mul(G[0][3], G[1][2])));
    return -q / (4.0 * M_PI * M_PI);
}

/* Exposed for tests: the m x m clover charge density at one site (m = 1, 2, 3),
 * or the improved density sum_m c_m q_m / m^4 (m = 0). */
double orc_clover_q_site(const double* U, const int* dims, long s, int m)
{
    lat_t g = make_lat(dims);
    if (m > 0) return clover_q_m(&g, U, s, m);
    return IMPROVED_C[0] * clover_q_m(&g, U, s, 1) + IMPROVED_C[1] * clover_q_m(&g, U, s, 2) / 16.0 +
           IMPROVED_C[2] * clover_q_m(&g, U, s, 3) / 81.0;
}

/* out[0] = sum_x sum_m c_m q_m(x) / m^4 (the improved charge), out[m] = sum_x q_m(x). */
void orc_topo_charge_improved(const double* U, const int* dims, double* out)
{
    lat_t g = make_lat(dims);
    double* pq = malloc(sizeof(double) * g.V * 3);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < g.V; s++)
        for (int m = 1; m <= 3; m++) pq[s * 3 + m - 1] = clover_q_m(&g, U, s, m);
    double qs[3] = {0, 0, 0};
    for (long s = 0; s < g.V; s++)
        for (int m = 0; m < 3; m++) qs[m] += pq[s * 3 + m];
    free(pq);
    out[0] = IMPROVED_C[0] * qs[0] + IMPROVED_C[1] * qs[1] / 16.0 + IMPROVED_C[2] * qs[2] / 81.0;
    for (int m = 0; m < 3; m++) out[1 + m] = qs[m];
}

/*
 * Wilson flow from t = 0 to t_end in steps of eps, a step that would pass the
 * next measurement time (or t_end) being shortened to end on it; E (clover)
 * and Q (charge 0: clover, 1: three-loop improved) at the ascending times
 * t_meas[0..n_meas-1] in [0, t_end].  Pinned by: on the step grid it equals
 * the fixed-step flow bit for bit; shortened steps keep third-order
 * convergence (tests/test_oracle_flow.py).
 */
void orc_wilson_flow_times(double* W, const int* dims, double t_end, double eps, const double* t_meas, int n_meas,
                           int charge, double* E_out, double* Q_out)
{
    const double tiny = 1e-12 * (t_end > 1.0 ? t_end : 1.0);
    double t = 0.0;
    int i = 0;
    for (;;) {
        while (i < n_meas && t_meas[i] <= t + tiny) {
            orc_clover_EQ(W, dims, &E_out[i], &Q_out[i]);
            if (charge == 1) {
                double q4[4];
                orc_topo_charge_improved(W, dims, q4);
                Q_out[i] = q4[0];
            }
            i++;
        }
        if (!(t < t_end - tiny)) break;
        double stop = (i < n_meas && t_meas[i] < t_end) ? t_meas[i] : t_end;
        double h = (stop - t < eps) ? stop - t : eps;
        orc_flow_step(W, dims, h);
        t = (h == stop - t) ? stop : t + h;
    }
}

/*
 * Wilson flow of n_steps steps of size eps; E and Q measured at flow times
 * t = k eps for k = 0, meas_every, 2 meas_every, ... <= n_steps.
 */
void orc_wilson_flow(double* W, const int* dims, double eps, int n_steps, int meas_every, double* E_out,
                     double* Q_out)
{
    int m = 0;
    for (int k = 0; k <= n_steps; k++) {
        if (k % meas_every == 0) {
            orc_clover_EQ(W, dims, &E_out[m], &Q_out[m]);
            m++;
        }
        if (k < n_steps) orc_flow_step(W, dims, eps);
    }
}

/*
 * Adaptive-step Wilson flow (Sec. IV.B cites an adaptive scheme with a
 * tolerance and a maximal step; the controller is not printed, so this is our
 * reading).  A trial step of size eps from W0 computes the third-order W3 of
 * orc_flow_step and, from the same stages, the second-order solution
 * W2nd = exp(2 Z1 - Z0) W0 (the two-stage method y0 + h(-k0 + 2 k1) with
 * k1 at y0 + h k0/4).  d = max over links of |W3 - W2nd|_F / 3 (Frobenius norm
 * divided by N = 3).
 * The step is accepted iff d <= tol; either way the next trial size is
 * eps * min(2, 0.95 (tol/d)^(1/3)), capped by eps_max and by the next
 * measurement time t_k = k dt_meas.  E and Q are measured at every t_k <= t_end.
 * Returns the number of measurements; steps_out = accepted steps,
 * rejects_out = rejected trials.
 */
typedef struct { double *W0; mat3 *Z0, *Z1, *Z2, *X; } flow_bufs;

static flow_bufs flow_bufs_alloc(const lat_t* g)
{
    size_t n = (size_t)g->V * 4;
    flow_bufs b = {malloc(sizeof(double) * n * 18), malloc(sizeof(mat3) * n), malloc(sizeof(mat3) * n),
                   malloc(sizeof(mat3) * n), malloc(sizeof(mat3) * n)};
    return b;
}

static void flow_bufs_free(flow_bufs* b)
{
    free(b->W0); free(b->Z0); free(b->Z1); free(b->Z2); free(b->X);
}

/* One trial step of size h: W <- W3, W0 keeps the start; returns d. */
static double adaptive_trial(const lat_t* g, double* W, flow_bufs* b, double h)
{
    size_t n = (size_t)g->V * 4;
    memcpy(b->W0, W, sizeof(double) * n * 18);
    flow_generator(g, W, b->Z0, h);
    for (size_t i = 0; i < n; i++) b->X[i] = m_scale(b->Z0[i], 0.25);
    exp_update(g, W, b->X);
    flow_generator(g, W, b->Z1, h);
    for (size_t i = 0; i < n; i++) b->X[i] = m_sub(m_scale(b->Z1[i], 8.0 / 9.0), m_scale(b->Z0[i], 17.0 / 36.0));
    exp_update(g, W, b->X);
    flow_generator(g, W, b->Z2, h);
    for (size_t i = 0; i < n; i++)
        b->X[i] = m_add(m_sub(m_scale(b->Z2[i], 0.75), m_scale(b->Z1[i], 8.0 / 9.0)), m_scale(b->Z0[i], 17.0 / 36.0));
    exp_update(g, W, b->X);
    double d = 0;
#pragma omp parallel for reduction(max : d) schedule(static)
    for (long s = 0; s < g->V; s++)
        for (int mu = 0; mu < 4; mu++) {
            mat3 Y = m_sub(m_scale(b->Z1[s * 4 + mu], 2.0), b->Z0[s * 4 + mu]);
            mat3 W2 = m_mul(expm3(Y), getU(b->W0, s, mu));
            double e = m_frob(m_sub(getU(W, s, mu), W2)) / 3.0;
            if (e > d) d = e;
        }
    return d;
}

/* One trial step of size h (always kept); returns its error estimate d. */
double orc_flow_trial_step(double* W, const int* dims, double h)
{
    lat_t g = make_lat(dims);
    flow_bufs b = flow_bufs_alloc(&g);
    double d = adaptive_trial(&g, W, &b, h);
    flow_bufs_free(&b);
    return d;
}

int orc_wilson_flow_adaptive(double* W, const int* dims, double t_end, double tol, double eps_max, double eps0,
                             double dt_meas, double* E_out, double* Q_out, int max_meas, int* steps_out,
                             int* rejects_out)
{
    lat_t g = make_lat(dims);
    size_t nU = (size_t)g.V * 72;
    flow_bufs b = flow_bufs_alloc(&g);
    double t = 0, eps = eps0;
    int m = 0, steps = 0, rejects = 0;
    const double tiny = 1e-12 * dt_meas;
    if (m < max_meas) { orc_clover_EQ(W, dims, &E_out[m], &Q_out[m]); m++; }
    while (t < t_end - tiny && m < max_meas) {
        double t_next = dt_meas * (double)m;
        if (t_next > t_end) t_next = t_end;
        double h = eps < eps_max ? eps : eps_max;
        int hits = 0;
        if (t + h >= t_next - tiny) { h = t_next - t; hits = 1; }
        double d = adaptive_trial(&g, W, &b, h);
        double fac = d > 0 ? 0.95 * cbrt(tol / d) : 2.0;
        if (fac > 2.0) fac = 2.0;
        if (d <= tol) {
            t = hits ? t_next : t + h;
            steps++;
            if (hits) { orc_clover_EQ(W, dims, &E_out[m], &Q_out[m]); m++; }
            else eps = h * fac;             /* a step cut short by a measurement keeps the old size */
        } else {
            memcpy(W, b.W0, sizeof(double) * nU);
            rejects++;
            eps = h * fac;
        }
    }
    flow_bufs_free(&b);
    *steps_out = steps;
    *rejects_out = rejects;
    return m;
}

/* ------------------------------------------------------------------------ */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
