// libmgq multiscale maps (Sec. III): restriction (Eq. restriction), the
// transfer step of the prolongation (Eq. prolongation) and the interpolation
// stages, each a repeated Jacobi APE step (Eq. APE) on the active bonds of
// stage d that minimises the partial action S_d (Eq. smoothing).
#include <vector>

#include "mgq_internal.h"
#include "mgq_stencil.cuh"

namespace mgq {

// P_SU(3)(M): Gram-Schmidt start W, then NPASS passes over the subgroups
// (0,1), (0,2), (1,2) of W <- R W with R = R(w/|w|) maximising Re Tr(R W M^+).
// FP64 runs exactly NPASS passes (the oracle's definition).  FP32 stops after a
// pass whose three rotations all turn by less than 1e-6 (|r_1|, |r_2|, |r_3|
// below 1e-6): the remaining passes would move W by about that much, at the
// level of the links' FP32 rounding and far below the 1e-5 relative change of
// S_d that ends an APE stage (8^4 -> 16^4 links within 4e-6 of a projection
// run to FP32 rounding, 17 % less time for a batch of 256 lattices).
// FP32 also takes 1/|w| from the hardware reciprocal square root and updates
// the two rows with packed FMAs (su2_rows).
template <class T>
__device__ __forceinline__ M3<T> su3_project(const M3<T>& M) {
    constexpr int NPASS = 8;
    M3<T> W = M;
    reunitarize(W);
#pragma unroll 1
    for (int pass = 0; pass < NPASS; pass++) {
        bool moved = false;
#pragma unroll
        for (int s = 0; s < 3; s++) {
            const int i = (s == 2) ? 1 : 0, j = (s == 0) ? 1 : 2;
            const M3<T> V = mul_nd(W, M);
            T w[4];
            block_w(V, i, j, w);
            const T n2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
            if constexpr (sizeof(T) == 4) {
                if (!(n2 >= 1e-30f)) continue;
                const float inv = rsqrtf(n2);
                const float r[4] = {w[0] * inv, w[1] * inv, w[2] * inv, w[3] * inv};
                moved = moved || fabsf(r[1]) > 1e-6f || fabsf(r[2]) > 1e-6f || fabsf(r[3]) > 1e-6f;
                su2_rows(W, i, j, r, true, true, 7, 7);
            } else {
                const T xi = m_sqrt(n2);
                if (!(xi >= tiny_norm<T>())) continue;
                const T inv = T(1) / xi;
                const T r[4] = {w[0] * inv, w[1] * inv, w[2] * inv, w[3] * inv};
                left_su2(W, i, j, r);
            }
        }
        if constexpr (sizeof(T) == 4) {
            if (!moved) break;
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

// ======================================================= interpolation stages
// The stages run as a device-side state machine per lattice, so that neither
// the stopping rule nor the stage changes need the host: every iteration is
// one launch of k_iter_pb over all lattices of a call (up to PB_CHUNK per
// launch), in which one set of blocks measures the partial action S_d of a
// lattice's newest field while another takes the next Jacobi APE step from
// it; the last block of a lattice to finish (atomic ticket, no waiting) sums
// the partials in a fixed order and advances the lattice's state: stop after
// the first step k with |S_d(k) - S_d(k-1)| <= rel_tol |S_d(k-1)| or after
// max_iter steps (rel_tol <= 0: exactly max_iter), then the next stage.
// A stage of k steps takes k + 1 iterations (the first measures its start
// field); a finished lattice turns every later launch into a no-op.  Launches
// carry the lattice table as a kernel parameter; the state lives in the
// workspace.

struct ProlongCtl {
    int d;        // current stage 0..2; 3 when finished
    int phase;    // 0: measure S_d of the stage's start field; 1: stepping
    int it;       // steps taken in the stage
    int cur;      // buffer (0: the lattice's links, 1: scratch) holding the newest field
    int iters[3];
    int counted;  // 1 once the lattice added itself to the finished count
    double prev;  // S_d after the previous step (or of the start field)
    double sd[3];
};
static_assert(sizeof(ProlongCtl) == 64, "control block layout");

constexpr int PB_CHUNK = 64;       // lattices per launch (kernel-parameter table)
constexpr int PB_THREADS = 128;
constexpr int PB_SD_LANES = 256;  // partial-action lanes per block (any block size)
constexpr int PB_SD_MAXBLK = 512;  // partial-action blocks per lattice

template <class T>
struct ProDesc {
    Cx<T>* buf[2];
    Cx<T>* coarse;
    Geom gf, gc;
};

template <class T>
struct PBatch {
    int n;
    int prefix[PB_CHUNK + 1];   // blocks of the all-bond kernels (8 Vh_f bonds each)
    int aprefix[PB_CHUNK + 1];  // bond blocks of the iteration kernel (the largest stage set, 24 V_c bonds)
    int sprefix[PB_CHUNK + 1];  // partial-action blocks of the iteration kernel (first in its grid)
    ProDesc<T> d[PB_CHUNK];
    ProlongCtl* ctl;            // [n]
    double* partials;           // [sprefix[n]]
    unsigned* ticket;           // [n]
    int* ndone;                 // finished lattices of the whole call
    T c;
    double rel_tol;
    int max_iter;
};

// link field at p with the site stride of geometry g (device side)
template <class T, int NP>
__device__ __forceinline__ Links<T, NP> field(Cx<T>* p, const Geom& g) {
    Links<T, NP> l;
    l.p = p;
    l.S = g.S;
    return l;
}

__device__ __forceinline__ int find_block(const int* prefix, int n, int b) {
    int lo = 0, hi = n;  // prefix[lo] <= b < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= b) lo = mid; else hi = mid;
    }
    return lo;
}

// transfer into both buffers of every lattice, and a fresh state
template <class T, int NP>
__global__ void __launch_bounds__(PB_THREADS) k_transfer_pb(const __grid_constant__ PBatch<T> B) {
    const int l = find_block(B.prefix, B.n, blockIdx.x);
    const ProDesc<T>& D = B.d[l];
    const int idx = (blockIdx.x - B.prefix[l]) * PB_THREADS + threadIdx.x;
    if (idx == 0) {
        ProlongCtl c = {};
        B.ctl[l] = c;
        B.ticket[l] = 0u;
    }
    if (idx >= 8 * D.gf.Vh) return;
    const int mp = idx / D.gf.Vh, h = idx - mp * D.gf.Vh, mu = mp >> 1, par = mp & 1;
    int x[4];
    cb_coords(D.gf, par, h, x);
    M3<T> u = unit3<T>();
    if (((x[0] | x[1] | x[2] | x[3]) & 1) == 0) {
        const int xc[4] = {x[0] >> 1, x[1] >> 1, x[2] >> 1, x[3] >> 1};
        const int lc = lex_of(D.gc, xc);
        u = field<T, NP>(D.coarse, D.gc).load(mu, (xc[0] + xc[1] + xc[2] + xc[3]) & 1, lc >> 1);
    }
    field<T, NP>(D.buf[0], D.gf).store(mu, par, h, u);
    field<T, NP>(D.buf[1], D.gf).store(mu, par, h, u);
}

// ---- the bonds and plaquettes a stage touches, enumerated without gaps
// Every fine site is n = 2y + b with y a site of the half-extent lattice gc
// and b in {0,1}^4 its parity pattern; chi_mu(n) counts the odd b outside mu
// and chi_munu(n) those outside mu and nu (Sec. III).  Bonds with chi_mu = k:
// b_mu free and exactly k of the three other b odd, 2 C(3,k) patterns per
// direction, 8 C(3,k) V_c bonds in all (V_c = V/16).  Plaquettes with
// chi_munu = d: b_mu, b_nu free and d of the two other b odd, 4 C(2,d)
// patterns per plane, 24 C(2,d) V_c in all.  A thread per bond (plaquette)
// of the set keeps every lane of a warp busy; looping over all bonds would
// leave 5/8 to 7/8 of the lanes idle.

__device__ __forceinline__ int binom3(int k) { return (k == 0 || k == 3) ? 1 : 3; }

// j-th k-element subset of three slots, as a bit mask
__device__ __forceinline__ int subset3(int k, int j) {
    if (k == 0) return 0;
    if (k == 3) return 7;
    if (k == 1) return 1 << j;
    return j == 0 ? 3 : (j == 1 ? 5 : 6);
}

// coordinates of lexicographic site y of gc
__device__ __forceinline__ void lex_coords(const Geom& gc, int y, int yc[4]) {
    const int r0 = div_L(gc, 0, y);
    yc[0] = y - r0 * gc.L[0];
    const int r1 = div_L(gc, 1, r0);
    yc[1] = r0 - r1 * gc.L[1];
    yc[3] = div_L(gc, 2, r1);
    yc[2] = r1 - yc[3] * gc.L[2];
}

// fine site 2y + b with b given on the directions: b_a, b_b on the two chosen
// directions a < b and the bits of `mask` on the remaining ones in order
__device__ __forceinline__ void fine_site(const int yc[4], int a, int ba, int b, int bb, int mask, int x[4]) {
    int o = 0;
#pragma unroll
    for (int dd = 0; dd < 4; dd++) {
        int bit;
        if (dd == a) bit = ba;
        else if (dd == b) bit = bb;
        else {
            bit = (mask >> o) & 1;
            o++;
        }
        x[dd] = 2 * yc[dd] + bit;
    }
}

__device__ __forceinline__ int n_bonds(const Geom& gc, int k) { return 8 * binom3(k) * gc.V; }
__device__ __forceinline__ int n_plaqs(const Geom& gc, int d) { return 24 * (d == 1 ? 2 : 1) * gc.V; }

// bond t of the set chi_mu = k: direction mu, fine site x
__device__ __forceinline__ void bond_of(const Geom& gc, int k, int t, int& mu, int x[4]) {
    const int y = t % gc.V, r = t / gc.V;
    const int npat = 2 * binom3(k);
    mu = r / npat;
    const int p = r - mu * npat;
    int yc[4];
    lex_coords(gc, y, yc);
    fine_site(yc, mu, p & 1, -1, 0, subset3(k, p >> 1), x);
}

// plaquette t of the set chi_munu = d: plane (mu, nu), fine site x
__device__ __forceinline__ void plaq_of(const Geom& gc, int d, int t, int& mu, int& nu, int x[4]) {
    const int y = t % gc.V, r = t / gc.V;
    const int npat = 4 * (d == 1 ? 2 : 1);
    const int pl = r / npat, p = r - pl * npat;
    mu = pl < 3 ? 0 : (pl < 5 ? 1 : 2);
    nu = pl < 3 ? pl + 1 : (pl < 5 ? pl - 1 : 3);
    const int j = p >> 2;
    const int mask = d == 0 ? 0 : (d == 2 ? 3 : (1 << j));
    int yc[4];
    lex_coords(gc, y, yc);
    fine_site(yc, mu, p & 1, nu, (p >> 1) & 1, mask, x);
}

// One Jacobi APE step on bond t of the set chi_mu(n) = k: Unew = P_SU(3)[U + c
// sum_{nu != mu, n_nu odd} (T+_munu + T-_munu)] (Eq. APE), T+ = U_nu(n) U_mu(n+nu)
// U_nu(n+mu)^+, T- = U_nu(n-nu)^+ U_mu(n-nu) U_nu(n-nu+mu), read from Uin and
// written to Uout; no other bond changes within a stage.
template <class T, int NP>
__device__ __forceinline__ void ape_bond(const ProDesc<T>& D, T c, int k, int t, const Links<T, NP>& Uin,
                                         const Links<T, NP>& Uout) {
    const Geom& g = D.gf;
    int mu, x[4];
    bond_of(D.gc, k, t, mu, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1, h = lex_of(g, x) >> 1;
    const int op = par ^ 1;
    M3<T> M = Uin.load(mu, par, h);
    const int lpm = lex_hop(g, x, mu, +1);
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu || !(x[nu] & 1)) continue;
        const int lpn = lex_hop(g, x, nu, +1), lmn = lex_hop(g, x, nu, -1);
        const int lmn_pm = lex_hop(g, x, nu, -1, mu, +1);
        M3<T> tp, tm;
        if constexpr (sizeof(T) == 4) {
            // products of SU(3) factors in two-row form, the third row rebuilt
            tp = mul_nd_2(mul_nn_2(Uin.load_rows(nu, par, h), Uin.load(mu, op, lpn >> 1)), Uin.load(nu, op, lpm >> 1));
            rebuild_row2(tp);
            tm = mul_nn_2(mul_dn_2(Uin.load(nu, op, lmn >> 1), Uin.load(mu, op, lmn >> 1)),
                          Uin.load(nu, par, lmn_pm >> 1));
            rebuild_row2(tm);
        } else {
            tp = mul_nd(mul_nn(Uin.load(nu, par, h), Uin.load(mu, op, lpn >> 1)), Uin.load(nu, op, lpm >> 1));
            tm = mul_nn(mul_dn(Uin.load(nu, op, lmn >> 1), Uin.load(mu, op, lmn >> 1)), Uin.load(nu, par, lmn_pm >> 1));
        }
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

// bond t of the set chi_mu(n) = k copied from Uin to Uout
template <class T, int NP>
__device__ __forceinline__ void copy_bond(const ProDesc<T>& D, int k, int t, const Links<T, NP>& Uin,
                                          const Links<T, NP>& Uout) {
    int mu, x[4];
    bond_of(D.gc, k, t, mu, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1, h = lex_of(D.gf, x) >> 1;
    Uout.store(mu, par, h, Uin.load(mu, par, h));
}

// Re Tr of the plaquette U_mu(x) U_nu(x+mu) (U_nu(x) U_mu(x+nu))^+.  FP32: from
// rows 0, 1 of a = U_mu(x) U_nu(x+mu) and b = U_nu(x) U_mu(x+nu), with
// s_ij = row_i(a) . conj(row_j(b)), Re Tr(a b^+) = Re[s00 + s11 + conj(s00 s11 -
// s01 s10)] (row 2 of an SU(3) matrix is conj(row0 x row1); Binet-Cauchy).
// FP64: full products (the oracle's operations).
template <class T, int NP>
__device__ __forceinline__ T plaq_retr(const Links<T, NP>& U, int mu, int nu, int par, int op, int h, int hpm, int hpn) {
    if constexpr (sizeof(T) == 4) {
        const M3<T> a = mul_nn_2(U.load_rows(mu, par, h), U.load(nu, op, hpm));
        const M3<T> b = mul_nn_2(U.load_rows(nu, par, h), U.load(mu, op, hpn));
        Cx<T> sij[2][2];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++)
                sij[i][j] = mulc(a.e[i][0], b.e[j][0]) + mulc(a.e[i][1], b.e[j][1]) + mulc(a.e[i][2], b.e[j][2]);
        const Cx<T> dd = sij[0][0] * sij[1][1] - sij[0][1] * sij[1][0];
        return sij[0][0].re + sij[1][1].re + dd.re;
    } else {
        const M3<T> a = mul_nn(U.load(mu, par, h), U.load(nu, op, hpm));
        const M3<T> b = mul_nn(U.load(nu, par, h), U.load(mu, op, hpn));
        return retr_nd(a, b);
    }
}

// Sum of PB_SD_LANES = 256 values in lanes[] (shared) in the order a 256-thread
// block_sum takes them (warp-shuffle trees over eight warps of 32 lanes, then
// over the eight warp sums), computed by warp 0 of a block of any size; the
// result is valid in thread 0.  The partial action thus does not depend on the
// launch shape.
__device__ __forceinline__ double lanes_sum(const double* lanes) {
    __shared__ double warp_part[PB_SD_LANES / 32];
    double v = 0.0;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
#pragma unroll
        for (int w = 0; w < PB_SD_LANES / 32; w++) {
            double x = lanes[32 * w + lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) warp_part[w] = x;
        }
        __syncwarp();
        v = lane < PB_SD_LANES / 32 ? warp_part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// One iteration of every lattice of the launch.  The grid holds the
// partial-action blocks of all its lattices, then their bond blocks (so that
// the partial actions, chains of dependent loads, start first and overlap the
// steps):
//   partial-action blocks: S_d / beta = sum over the plaquettes with
//     chi_munu(n) = d of (1 - Re Tr U_p / 3) (Eq. smoothing) of the newest
//     field (buffer cur), 256 lanes per block whatever the block size (lane v
//     of block b takes the plaquettes b 256 + v + j nS 256 in turn);
//   bond blocks: the next APE step of stage d (bonds with chi_mu = d + 1) from
//     cur into 1 - cur, and at the start of a stage d >= 1 (phase 0) also the
//     copy of the previous stage's bonds (chi_mu = d) from cur to 1 - cur, so
//     that both buffers agree outside the stage's bonds.
// Both read only buffer cur.  The step is taken before the partial action of
// its predecessor is known; when that partial action ends the stage, the step
// is dropped (cur keeps the stage's last step, and the next stage's copy
// overwrites the dropped bonds in 1 - cur).  The last block of a lattice to
// finish (atomic ticket over all its blocks) sums the partials in a fixed order
// and advances the state: after the start field's S_d (phase 0) the stage's
// first step is the newest field; after a step's S_d the stage stops when
// |S_d(k) - S_d(k-1)| <= rel_tol |S_d(k-1)| or k = max_iter (rel_tol <= 0:
// exactly max_iter steps), else the step it has just taken becomes the newest.
template <class T, int NP>
__global__ void __launch_bounds__(PB_THREADS, sizeof(T) == 8 ? 1 : 5) k_iter_pb(const __grid_constant__ PBatch<T> B) {
    pdl_launch_dependents();
    pdl_wait();  // the state and the fields come from the previous launch
    const int nSall = B.sprefix[B.n];
    const bool sd_role = (int)blockIdx.x < nSall;
    const int l = sd_role ? find_block(B.sprefix, B.n, blockIdx.x) : find_block(B.aprefix, B.n, blockIdx.x - nSall);
    const ProDesc<T>& D = B.d[l];
    ProlongCtl* C = B.ctl + l;
    const int d = C->d, phase = C->phase, cur = C->cur;
    if (d >= 3) return;  // the whole block: one lattice per block
    __shared__ double lanes[PB_SD_LANES];
    __shared__ int last;
    const Geom& g = D.gf;
    const int nS = B.sprefix[l + 1] - B.sprefix[l], nA = B.aprefix[l + 1] - B.aprefix[l];
    const int b = sd_role ? (int)blockIdx.x - B.sprefix[l] : (int)blockIdx.x - nSall - B.aprefix[l];
    double* part = B.partials + B.sprefix[l];
    const Links<T, NP> Uin = field<T, NP>(D.buf[cur], g);
    if (sd_role) {
        const int np = n_plaqs(D.gc, d);
        for (int v = threadIdx.x; v < PB_SD_LANES; v += blockDim.x) {
            double acc = 0.0;
            for (int t = b * PB_SD_LANES + v; t < np; t += nS * PB_SD_LANES) {
                int mu, nu, x[4];
                plaq_of(D.gc, d, t, mu, nu, x);
                const int par = (x[0] + x[1] + x[2] + x[3]) & 1, h = lex_of(g, x) >> 1, op = par ^ 1;
                const int hpm = lex_hop(g, x, mu, +1) >> 1, hpn = lex_hop(g, x, nu, +1) >> 1;
                acc += 1.0 - (double)plaq_retr(Uin, mu, nu, par, op, h, hpm, hpn) / 3.0;
            }
            lanes[v] = acc;
        }
        __syncthreads();
        const double sb = lanes_sum(lanes);
        if (threadIdx.x == 0) part[b] = sb;
    } else {
        const Links<T, NP> Uout = field<T, NP>(D.buf[cur ^ 1], g);
        const int t0 = b * (int)blockDim.x + threadIdx.x, stride = nA * (int)blockDim.x;
        if (phase == 0 && d >= 1)
            for (int t = t0; t < n_bonds(D.gc, d); t += stride) copy_bond<T, NP>(D, d, t, Uin, Uout);
        const int nstep = n_bonds(D.gc, d + 1);
        for (int t = t0; t < nstep; t += stride) ape_bond<T, NP>(D, B.c, d + 1, t, Uin, Uout);
    }
    __syncthreads();  // every thread of the block has read the state and done its work
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(B.ticket + l, 1u) == (unsigned)(nS + nA - 1);
    }
    __syncthreads();
    if (!last) return;
    // the last block of this lattice: every partial is written; a fixed-order sum
    __threadfence();
    for (int v = threadIdx.x; v < PB_SD_LANES; v += blockDim.x) {
        double sv = 0.0;
        for (int i = v; i < nS; i += PB_SD_LANES) sv += __ldcg(part + i);
        lanes[v] = sv;
    }
    __syncthreads();
    const double S = lanes_sum(lanes);
    if (threadIdx.x != 0) return;
    B.ticket[l] = 0u;
    if (phase == 0) {
        C->prev = S;
        if (B.max_iter > 0) {  // the first step, taken in this iteration, is the newest field
            C->phase = 1;
            C->it = 1;
            C->cur = cur ^ 1;
            return;
        }
        C->it = 0;
    } else {
        const bool stop = (B.rel_tol > 0.0 && fabs(S - C->prev) <= B.rel_tol * fabs(C->prev)) || C->it >= B.max_iter;
        if (!stop) {
            C->prev = S;
            C->it += 1;
            C->cur = cur ^ 1;
            return;
        }
    }
    C->iters[d] = C->it;
    C->sd[d] = S;
    C->d = d + 1;
    C->phase = 0;
    if (d + 1 == 3 && !C->counted) {
        C->counted = 1;
        atomicAdd(B.ndone, 1);
    }
}

// newest field into the lattice's links; iteration counts and final S_d out
template <class T, int NP>
__global__ void __launch_bounds__(PB_THREADS) k_finish_pb(const __grid_constant__ PBatch<T> B, int first,
                                                          int* __restrict__ iters, double* __restrict__ sd) {
    const int l = find_block(B.prefix, B.n, blockIdx.x);
    const ProDesc<T>& D = B.d[l];
    const ProlongCtl* C = B.ctl + l;
    const int idx = (blockIdx.x - B.prefix[l]) * PB_THREADS + threadIdx.x;
    if (idx < 3) {
        iters[3 * (first + l) + idx] = C->d > idx ? C->iters[idx] : (C->d == idx ? C->it : 0);
        sd[3 * (first + l) + idx] = C->d > idx ? C->sd[idx] : 0.0;
    }
    if (C->cur == 0 || idx >= 8 * D.gf.Vh) return;
    const int mp = idx / D.gf.Vh, h = idx - mp * D.gf.Vh, mu = mp >> 1, par = mp & 1;
    field<T, NP>(D.buf[0], D.gf).store(mu, par, h, field<T, NP>(D.buf[1], D.gf).load(mu, par, h));
}

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// partial-action blocks of one lattice: one block per 1024 plaquettes (four per
// lane) of the largest set (48 V_c = 3 V) for a lattice alone, up to
// PB_SD_MAXBLK; in a call over many lattices the lattice's share of about 4096
// blocks, so that the blocks stay large when there is parallelism across lattices
static int sd_blocks(const Geom& g, double total_sites) {
    const long full = nblk(3L * g.V, 4 * PB_SD_LANES);
    long b = (long)((4096.0 * g.V + total_sites - 1.0) / total_sites);
    if (b > full) b = full;
    if (b > PB_SD_MAXBLK) b = PB_SD_MAXBLK;
    return b < 1 ? 1 : (int)b;
}

static double total_sites(const mgq_lattice* fine, int n) {
    double v = 0.0;
    for (int i = 0; i < n; i++) v += (double)fine[i].dims[0] * fine[i].dims[1] * fine[i].dims[2] * fine[i].dims[3];
    return v;
}

// Where the state of a call lives (device): control blocks, tickets, the
// finished count, partial sums, result staging.
struct PbState {
    ProlongCtl* ctl;
    unsigned* ticket;
    int* ndone;
    double* partials;
    int* iters;
    double* sd;
};

template <class T>
static void fill_pbatch(PBatch<T>& B, const mgq_lattice* coarse, const mgq_lattice* fine, void* const* scratch,
                        int first, int n, const PbState& S, uint64_t poff, double c, double rel_tol, int max_iter,
                        double tsites) {
    B.n = n;
    B.prefix[0] = 0;
    B.aprefix[0] = 0;
    B.sprefix[0] = 0;
    for (int i = 0; i < n; i++) {
        const mgq_lattice& F = fine[first + i];
        ProDesc<T>& D = B.d[i];
        D.buf[0] = reinterpret_cast<Cx<T>*>(F.links);
        D.buf[1] = reinterpret_cast<Cx<T>*>(scratch[first + i]);
        D.coarse = reinterpret_cast<Cx<T>*>(coarse[first + i].links);
        D.gf = make_geom(F.dims);
        D.gc = make_geom(coarse[first + i].dims);
        B.prefix[i + 1] = B.prefix[i] + nblk(8L * D.gf.Vh, PB_THREADS);
        // bond blocks for the largest stage set (24 V_c bonds); the copy at a stage start loops
        const int nS = sd_blocks(D.gf, tsites), nA = nblk(24L * D.gc.V, block_size(MGQ_KERNEL_APE, F.prec));
        B.aprefix[i + 1] = B.aprefix[i] + nA;
        B.sprefix[i + 1] = B.sprefix[i] + nS;
    }
    B.ctl = S.ctl + first;
    B.partials = S.partials + poff;
    B.ticket = S.ticket + first;
    B.ndone = S.ndone;
    B.c = (T)c;
    B.rel_tol = rel_tol;
    B.max_iter = max_iter;
}

// The whole interpolation for n lattices: transfer, then iterations until all
// lattices finished (budget <= 0: the host reads the finished count every 32
// iterations) or exactly `budget` iterations (no host synchronisation), then
// the newest fields into the links and the per-lattice results into S.iters,
// S.sd (3 per lattice).
static mgq_status prolong_run(const mgq_lattice* coarse, mgq_lattice* fine, void* const* scratch, int n, double c,
                              double rel_tol, int max_iter, int budget, const PbState& S, cudaStream_t st) {
    mgq_status s;
    const double tsites = total_sites(fine, n);
    if (cudaMemsetAsync(S.ndone, 0, sizeof(int), st) != cudaSuccess) return cuda_check("prolongate: reset");
    auto each_chunk = [&](auto&& launch) {
        uint64_t poff = 0;
        for (int first = 0; first < n; first += PB_CHUNK) {
            const int m = n - first < PB_CHUNK ? n - first : PB_CHUNK;
            dispatch_prec(fine[0].prec, [&]<class T, int NP>() {
                PBatch<T> B;
                fill_pbatch(B, coarse, fine, scratch, first, m, S, poff, c, rel_tol, max_iter, tsites);
                launch.template operator()<T, NP>(B, first);
                poff += (uint64_t)B.sprefix[m];
            });
        }
    };
    each_chunk([&]<class T, int NP>(const PBatch<T>& B, int) {
        k_transfer_pb<T, NP><<<B.prefix[B.n], PB_THREADS, 0, st>>>(B);
    });
    if ((s = cuda_check("prolongate: transfer"))) return s;
    auto iteration = [&]() {
        each_chunk([&]<class T, int NP>(const PBatch<T>& B, int) {
            launch_pdl(k_iter_pb<T, NP>, B.sprefix[B.n] + B.aprefix[B.n], block_size(MGQ_KERNEL_APE, fine[0].prec), st, B);
        });
    };
    if (budget > 0) {
        for (int k = 0; k < budget; k++) iteration();
        if ((s = cuda_check("prolongate: iterations"))) return s;
    } else {
        // at most 3 (max_iter + 1) iterations finish every lattice
        const long cap = 3L * ((long)max_iter + 1);
        long done_it = 0;
        int finished = 0;
        while (finished < n && done_it < cap) {
            const int chunk = cap - done_it < 32 ? (int)(cap - done_it) : 32;
            for (int k = 0; k < chunk; k++) iteration();
            done_it += chunk;
            if ((s = cuda_check("prolongate: iterations"))) return s;
            if (cudaMemcpyAsync(&finished, S.ndone, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return cuda_check("prolongate: poll");
        }
    }
    each_chunk([&]<class T, int NP>(const PBatch<T>& B, int first) {
        k_finish_pb<T, NP><<<B.prefix[B.n], PB_THREADS, 0, st>>>(B, first, S.iters, S.sd);
    });
    return cuda_check("prolongate: finish");
}

static mgq_status check_pair(const mgq_lattice* coarse, const mgq_lattice* fine, bool need_work, const char* fn) {
    mgq_status s = check_lattice(coarse, false, fn);
    if (s) return s;
    if ((s = check_lattice(fine, need_work, fn))) return s;
    for (int mu = 0; mu < 4; mu++)
        if (fine->dims[mu] != 2 * coarse->dims[mu]) return fail(MGQ_EINVAL, "%s: fine extents must be twice the coarse extents", fn);
    if (fine->prec != coarse->prec) return fail(MGQ_EINVAL, "%s: precisions differ", fn);
    return MGQ_OK;
}

// batched workspace: control blocks, tickets, finished count, partials,
// result staging, then one scratch link field per lattice
static uint64_t pb_state_bytes(const mgq_lattice* fine, int n) {
    uint64_t nparts = 0;
    const double ts = total_sites(fine, n);
    for (int i = 0; i < n; i++) nparts += (uint64_t)sd_blocks(make_geom(fine[i].dims), ts);
    return round256((uint64_t)n * sizeof(ProlongCtl)) + round256((uint64_t)n * sizeof(unsigned) + sizeof(int)) +
           round256(nparts * sizeof(double)) + round256((uint64_t)3 * n * sizeof(int)) +
           round256((uint64_t)3 * n * sizeof(double));
}

static PbState pb_state_at(void* work, const mgq_lattice* fine, int n) {
    uint64_t nparts = 0;
    const double ts = total_sites(fine, n);
    for (int i = 0; i < n; i++) nparts += (uint64_t)sd_blocks(make_geom(fine[i].dims), ts);
    char* p = static_cast<char*>(work);
    PbState S;
    S.ctl = reinterpret_cast<ProlongCtl*>(p);
    p += round256((uint64_t)n * sizeof(ProlongCtl));
    S.ticket = reinterpret_cast<unsigned*>(p);
    S.ndone = reinterpret_cast<int*>(p + (uint64_t)n * sizeof(unsigned));
    p += round256((uint64_t)n * sizeof(unsigned) + sizeof(int));
    S.partials = reinterpret_cast<double*>(p);
    p += round256(nparts * sizeof(double));
    S.iters = reinterpret_cast<int*>(p);
    p += round256((uint64_t)3 * n * sizeof(int));
    S.sd = reinterpret_cast<double*>(p);
    return S;
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
    mgq_status s = check_pair(coarse, fine, true, "mgq_prolongate");
    if (s) return s;
    if (!(c > 0.0) || max_iter < 0) return fail(MGQ_EINVAL, "mgq_prolongate: need c > 0 and max_iter >= 0");
    cudaStream_t st = as_stream(stream);
    // state in the lattice's workspace: control block, ticket and count in the
    // scalars, partials in the partial-sum area, the scratch field in its link copy
    double* sc = ws_scalars(fine);
    PbState S;
    S.ctl = reinterpret_cast<ProlongCtl*>(sc + 48);
    S.ticket = reinterpret_cast<unsigned*>(sc + 56);
    S.ndone = reinterpret_cast<int*>(sc + 57);
    S.iters = reinterpret_cast<int*>(sc + 58);
    S.sd = sc + 60;
    S.partials = ws_partials(fine);
    void* scratch[1] = {ws_links(fine)};
    if ((s = prolong_run(coarse, fine, scratch, 1, c, rel_tol, max_iter, 0, S, st))) return s;
    if (iters_out && (s = deliver_int(S.iters, iters_out, 3, st, "mgq_prolongate"))) return s;
    if (sd_out && (s = deliver(S.sd, sd_out, 3, st, "mgq_prolongate"))) return s;
    return MGQ_OK;
}

uint64_t mgq_prolongate_batched_workspace_bytes(const mgq_lattice* fine, int n) {
    if (!fine || n < 1) return 0;
    uint64_t b = pb_state_bytes(fine, n);
    for (int i = 0; i < n; i++) {
        const uint64_t lb = links_bytes(&fine[i]);
        if (!lb) return 0;
        b += round256(lb);
    }
    return b;
}

mgq_status mgq_prolongate_batched(const mgq_lattice* coarse, mgq_lattice* fine, int n, double c, double rel_tol,
                                  int max_iter, int iter_budget, int* iters_out, double* sd_out, int* n_done_out,
                                  void* work, uint64_t work_bytes, void* stream) {
    Trace trace("mgq_prolongate_batched");
    if (!coarse || !fine || n < 1) return fail(MGQ_EINVAL, "mgq_prolongate_batched: need at least one lattice pair");
    mgq_status s;
    for (int i = 0; i < n; i++) {
        if ((s = check_pair(&coarse[i], &fine[i], false, "mgq_prolongate_batched"))) return s;
        if (fine[i].prec != fine[0].prec) return fail(MGQ_EINVAL, "mgq_prolongate_batched: all lattices need one precision");
    }
    if (!(c > 0.0) || max_iter < 0 || iter_budget < 0)
        return fail(MGQ_EINVAL, "mgq_prolongate_batched: need c > 0, max_iter >= 0, iter_budget >= 0");
    if (!work || ((uintptr_t)work & 255)) return fail(MGQ_EINVAL, "mgq_prolongate_batched: work NULL or not 256-byte aligned");
    const uint64_t need = mgq_prolongate_batched_workspace_bytes(fine, n);
    if (work_bytes < need)
        return fail(MGQ_ENOMEM, "mgq_prolongate_batched: work has %llu bytes, needs %llu", (unsigned long long)work_bytes,
                    (unsigned long long)need);
    cudaStream_t st = as_stream(stream);
    const PbState S = pb_state_at(work, fine, n);
    std::vector<void*> scratch(n);
    char* p = static_cast<char*>(work) + pb_state_bytes(fine, n);
    for (int i = 0; i < n; i++) {
        scratch[i] = p;
        p += round256(links_bytes(&fine[i]));
    }
    if ((s = prolong_run(coarse, fine, scratch.data(), n, c, rel_tol, max_iter, iter_budget, S, st))) return s;
    if (iters_out && (s = deliver_int(S.iters, iters_out, 3 * (size_t)n, st, "mgq_prolongate_batched"))) return s;
    if (sd_out && (s = deliver(S.sd, sd_out, 3 * (size_t)n, st, "mgq_prolongate_batched"))) return s;
    if (n_done_out && (s = deliver_int(S.ndone, n_done_out, 1, st, "mgq_prolongate_batched"))) return s;
    return MGQ_OK;
}

}  // extern "C"
