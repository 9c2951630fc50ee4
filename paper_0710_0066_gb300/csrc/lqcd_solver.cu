// lqcd_solver.cu -- persistent batched solver for the even-odd reduced
// operator  A = 1 - kappa^2 H_eo H_oe  on a batch of independent systems:
// every x0-slab of one colour (W1 restricted to the slab, Sec. 1) or the
// whole lattice (M, the S4 solver of Sec. 3).
//
// One cooperative launch runs the whole solve:
//   outer loop (double):  r = b - A x, stop when |r| <= tol |b| per system;
//   inner loop (double, single or half storage, FP32 arithmetic):
//     BiCGstab on A e = r / |r| to a relative residual inner_tol;
//   x += |r| e.
// Each system is handled by its own group of CTAs (cps CTAs per system).
// Reductions are per system, in double, in a fixed order (warp shuffles,
// then the group's per-CTA partials summed in CTA order), so every CTA of a
// group computes bitwise the same scalars and takes the same decisions.
// The systems never wait for one another: a group meets only at its own
// software barrier (one counter per system), loops until its own system has
// converged and returns; the kernel ends when every group has.  The barrier
// wait is bounded (about two seconds unless lqcd_set_wait_limit says
// otherwise): on time-out the kernel records LQCD_ERR_TIMEOUT and every CTA
// returns at its next barrier.
#include <stdio.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "lqcd_common.cuh"

namespace {

constexpr int SBS = 256;
// the hopping term's loop over the directions stays rolled inside the
// persistent solver: its phases together would not fit the instruction
// cache with every hop specialised (a build option; 4 unrolls it)
#ifndef LQCD_SOLVE_UNR
#define LQCD_SOLVE_UNR 1
#endif
constexpr int SOLVE_UNR = LQCD_SOLVE_UNR;
// the geometric series (and the Schwarz preconditioner built from it) is a
// two-phase loop whose code fits the cache: it keeps every hop specialised
// (measured at 16^3 x 32: rolled BiCGstab 11 % faster, rolled series 10 %
// slower)
constexpr int SERIES_UNR = 4;
constexpr int NSYS_MAX = 64;
constexpr int NQ = 3;
constexpr int NACC = 5;  // iteration sums kept beside the sticky status

// per-system state codes in the flag arrays
enum { F_ACTIVE = 0, F_DONE = 1, F_NAN = 2, F_MAXIT = 3 };

struct SolveArgs {
    Geo g;
    int mode;  // MODE_INTRA: slabs, MODE_ALL: whole lattice
    double k2;
    double diag;  // the system is diag - k2 H_eo H_oe (1, or 1 + rho for W3,eo)
    int method;   // SOLVER_BICGSTAB or SOLVER_SERIES (inner iteration)
    int guess;    // 1: x holds an initial guess on entry, 0: start from x = 0
    int nsys, cps;
    int chunk;  // sites of one system handled by one CTA (the last CTA may get fewer)
    int slab0, slabstep;
    int nsite;
    GaugeF U64, UP;
    SpinorF b, x, r64;  // double, parity 0
    SpinorF t64;        // parity 1: double (double solve) or df pairs (mixed)
    SpinorF r, rh, p, v, s, t;  // inner precision, parity 0
    SpinorF tmp;        // inner precision, parity 1
    SpinorF e;          // inner solution (single; double for the double solver)
    double tol, inner_tol;
    int max_iter, max_outer, max_inner;
    double* part;       // [NQ][grid]
    unsigned* bar;      // one barrier counter per system, BAR_STRIDE apart
    int* status;
    int* sticky;        // first failure of any solve since the host last read it
    unsigned long long* acc;  // [5] inner iterations, BiCGstab iterations x sites,
                              // outer cycles x sites, series iterations x sites,
                              // Schwarz-preconditioned iterations x sites
    int* iters;         // [nsys]
    double* resid;      // [nsys]
    int* outer_out;
    long long spin_limit;  // clock64 cycles of one barrier wait before LQCD_ERR_TIMEOUT
    // Schwarz-preconditioned inner solve of the whole lattice (SOLVER_SAP):
    // full-lattice vectors in the inner precision, [0] the even, [1] the odd
    // parity block; fy (the inner solution) in the precision of e, whose
    // even block it is
    double kappa;
    int nsap;  // geometric-series terms of every block solve of the preconditioner
    // SOLVER_SAPB: 4-D Schwarz blocks of extents bk[mu] (2 or 4, lbk = log2),
    // nbk[mu] = L[mu] / bk[mu] blocks per direction, nblk in all, bvh sites
    // of one parity in a block
    int bk[4], lbk[4], nbk[4], nblk, bvh;
    SpinorF fr[2], frh[2], fp[2], fv[2], fs[2], ft[2], fzp[2], fzs[2], fw1[2], fw2[2], fy[2];
};

struct SysSt {  // the CTA's own system
    double bn2, rn2, rr, itol2;
    double2 rho, alpha, omega, beta;
    int active, idone, it, itc, flag;
};

// barrier counters of different systems sit on different 128-byte lines
constexpr int BAR_STRIDE = 32;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// barrier over the cps CTAs of one system (the systems are independent and
// never wait for one another); bounded: gives up after A.spin_limit cycles
__device__ bool sys_sync(const SolveArgs& A, int sys, unsigned& epoch)
{
    __shared__ int s_bad;
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        unsigned* bar = A.bar + (size_t)sys * BAR_STRIDE;
        const unsigned target = epoch * (unsigned)A.cps;
        __threadfence();
        atomicAdd(bar, 1u);
        const long long t0 = clock64();
        int bad = 0;
        while (ld_acquire(bar) < target) {
            if (*(volatile int*)A.status == LQCD_ERR_TIMEOUT) { bad = 1; break; }
            if (clock64() - t0 > A.spin_limit) {
                atomicExch(A.status, LQCD_ERR_TIMEOUT);
                atomicCAS(A.sticky, 0, LQCD_ERR_TIMEOUT);
                bad = 1;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_bad = bad;
    }
    __syncthreads();
    return s_bad == 0;
}

// CTA sum of up to three doubles -> part[rb][q][cta].  The partials are
// double-buffered (rb alternates with every gather): a CTA that starts the
// next reduction while a slower CTA of its system still reads the previous
// one writes the other buffer, and the barrier inside every put / gather
// pair keeps the reuse of a buffer two reductions later safe.
__device__ void reduce_put(const SolveArgs& A, double a, double b, double c, int nq, int rb)
{
    __shared__ double sh[NQ][SBS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
        sh[2][w] = c;
    }
    __syncthreads();
    if ((int)threadIdx.x < nq) {
        double v = 0.0;
        for (int k = 0; k < SBS / 32; ++k) v += sh[threadIdx.x][k];
        A.part[((size_t)rb * NQ + threadIdx.x) * gridDim.x + blockIdx.x] = v;
    }
}

// totals of the own system's partials: warp q sums quantity q
__device__ void gather_own(const SolveArgs& A, int sys, int nq, double* out, int& rb)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < nq) {
        const double* p = A.part + ((size_t)rb * NQ + w) * gridDim.x + (size_t)sys * A.cps;
        double v = 0.0;
        for (int c = lane; c < A.cps; c += 32) v += p[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) out[w] = v;
    }
    rb ^= 1;
    __syncthreads();
}

// per-site dot products in the storage arithmetic (T), accumulated over the
// sites of a thread and across threads in double
template <class T>
__device__ __forceinline__ void cdot_acc(const Spinor<T>& a, const Spinor<T>& b, double& re, double& im)
{
    T sr = 0, si = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sr += a.c[s][c].re * b.c[s][c].re + a.c[s][c].im * b.c[s][c].im;
            si += a.c[s][c].re * b.c[s][c].im - a.c[s][c].im * b.c[s][c].re;
        }
    re += (double)sr;
    im += (double)si;
}
template <class T>
__device__ __forceinline__ double nrm_acc(const Spinor<T>& a)
{
    T r = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) r += a.c[s][c].re * a.c[s][c].re + a.c[s][c].im * a.c[s][c].im;
    return (double)r;
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b)
{
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// sites of a system are split into contiguous chunks, one per CTA
#define FOR_SITES                                                                                   \
    for (int j_ = cin * A.chunk + (int)threadIdx.x, je_ = min(A.nsite, (cin + 1) * A.chunk); j_ < je_; \
         j_ += SBS)
// element-wise phases of the single-precision inner solver run over 16-byte
// words (one float4 = two complex components) instead of whole sites: six
// times the parallelism and few live registers per thread
#define FOR_WORDS for (int f_ = cin * SBS + (int)threadIdx.x; f_ < 6 * A.nsite; f_ += A.cps * SBS)
#define WORD_ADDR const size_t a = (size_t)(f_ / A.nsite) * A.g.Vh + base + (f_ % A.nsite)
#define W4(f) ((float4*)(f).v)
#define SYNC_OR_RETURN \
    if (!sys_sync(A, sys, epoch)) return

// y + a x for the two complex numbers of a word
__device__ __forceinline__ float4 caxpy2(float2 a, float4 x, float4 y)
{
    return make_float4(y.x + a.x * x.x - a.y * x.y, y.y + a.x * x.y + a.y * x.x, y.z + a.x * x.z - a.y * x.w,
                       y.w + a.x * x.w + a.y * x.z);
}
// word-parallel dot products: each thread sums its few words in FP32 and
// hands the sum to the FP64 reduction once (GB300 issues FP64 at a small
// fraction of the FP32 rate; the single-precision inner solver's scalars
// need no more than FP32 accuracy per thread)
__device__ __forceinline__ void cdot2(float4 a, float4 b, float& re, float& im)
{
    re += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    im += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
}
__device__ __forceinline__ float nrm2w(float4 a) { return a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w; }

// single-precision spinor at site j of the combination y + a x of two
// inner vectors (word by word, as the element-wise phases form it), and of
// y + b (z + a x) of three
__device__ __forceinline__ void load_axpy32(const SpinorF& x, const SpinorF& y, float2 a, int j, Spinor<float>& s)
{
    const float4* xp = (const float4*)x.v;
    const float4* yp = (const float4*)y.v;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 w = caxpy2(a, xp[(size_t)k * x.N + j], yp[(size_t)k * y.N + j]);
        s.c[(2 * k) / 3][(2 * k) % 3] = mk(w.x, w.y);
        s.c[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(w.z, w.w);
    }
}
__device__ __forceinline__ void load_axpypz32(const SpinorF& x, const SpinorF& z, const SpinorF& y, float2 a, float2 b,
                                              int j, Spinor<float>& s)
{
    const float4* xp = (const float4*)x.v;
    const float4* zp = (const float4*)z.v;
    const float4* yp = (const float4*)y.v;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const size_t o = (size_t)k * x.N + j;
        const float4 w = caxpy2(b, caxpy2(a, xp[o], zp[o]), yp[o]);
        s.c[(2 * k) / 3][(2 * k) % 3] = mk(w.x, w.y);
        s.c[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(w.z, w.w);
    }
}

template <class T>
__device__ __forceinline__ void sp_axpy(Spinor<T>& y, T a, const Spinor<T>& x)  // y <- x + a y
{
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) y.c[s][c] = x.c[s][c] + a * y.c[s][c];
}
template <class T>
__device__ __forceinline__ void sp_zero(Spinor<T>& y)
{
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) y.c[s][c] = mk(T(0), T(0));
}

// eo index of the t-th site of one parity in the slabs of colour c
// (t < Vh / 2): slab 2k + c holds eo indices [(2k + c) Sh, (2k + c + 1) Sh)
__device__ __forceinline__ int colour_site(const Geo& g, int c, int t)
{
    const int k = t / g.Sh;
    return (c + 2 * k) * g.Sh + (t - k * g.Sh);
}

#define SAP_SYNC \
    if (!sys_sync(A, sys, epoch)) return false
#define FOR_COLOUR_SITES(c) \
    for (int t_ = cin * SBS + (int)threadIdx.x, i = 0; t_ < A.g.Vh / 2 && ((i = colour_site(A.g, (c), t_)), true); \
         t_ += A.cps * SBS)

// z = K^-1 q, the Schwarz preconditioner of the global solve (Sec. 3, S4
// solver): one multiplicative cycle over the x0-slabs, first the red slabs
// (z_r = A^-1 q_r), then the black ones with the source corrected by the
// hops from the red faces (z_b = D^-1 (q_b + kappa H_cross z_r)).  Every slab
// solve is the even-odd reduced slab operator 1 - kappa^2 H_eo H_oe inverted
// by nsap terms of its geometric series (the paper's block solver), so K^-1
// is a fixed polynomial in the operators: a linear preconditioner, as
// BiCGstab needs.  Full-lattice vectors in P; 4 nsap + 5 barriers.
template <int P>
__device__ bool sap_apply(const SolveArgs& A, int sys, int cin, unsigned& epoch, const SpinorF* q, const SpinorF* z)
{
    typedef typename Real<P>::T T;
    const T kap = (T)A.kappa, k2 = (T)A.k2;
    for (int c = 0; c < 2; ++c) {
        const SpinorF* src = c == 0 ? q : A.fw2;
        // be_e = src_e + kappa H_eo src_o on the slabs of colour c; u_0 = be
        FOR_COLOUR_SITES(c)
        {
            Spinor<T> a, b;
            hop_site<P, false, SERIES_UNR>(A.g, MODE_INTRA, 0, 0, i, src[1], A.UP, a);
            load_spinor<P, false>(src[0], i, b);
            sp_axpy(a, kap, b);
            store_spinor<P>(A.fw1[0], i, a);
            store_spinor<P>(z[0], i, a);
        }
        SAP_SYNC;
        for (int n = 0; n < A.nsap; ++n) {
            // w1_o = H_oe u_e
            FOR_COLOUR_SITES(c)
            {
                Spinor<T> a;
                hop_site<P, false, SERIES_UNR>(A.g, MODE_INTRA, 0, 1, i, z[0], A.UP, a);
                store_spinor<P>(A.fw1[1], i, a);
            }
            SAP_SYNC;
            // u_e = be_e + kappa^2 H_eo w1_o
            FOR_COLOUR_SITES(c)
            {
                Spinor<T> a, b;
                hop_site<P, false, SERIES_UNR>(A.g, MODE_INTRA, 0, 0, i, A.fw1[1], A.UP, a);
                load_spinor<P, false>(A.fw1[0], i, b);
                sp_axpy(a, k2, b);
                store_spinor<P>(z[0], i, a);
            }
            SAP_SYNC;
        }
        // z_o = src_o + kappa H_oe u_e
        FOR_COLOUR_SITES(c)
        {
            Spinor<T> a, b;
            hop_site<P, false, SERIES_UNR>(A.g, MODE_INTRA, 0, 1, i, z[0], A.UP, a);
            load_spinor<P, false>(src[1], i, b);
            sp_axpy(a, kap, b);
            store_spinor<P>(z[1], i, a);
        }
        SAP_SYNC;
        if (c == 0) {
            // black source: w2 = q + kappa H_cross z_r (non-zero hops only on
            // the slab faces), both parities
            for (int t_ = cin * SBS + (int)threadIdx.x; t_ < A.g.Vh; t_ += A.cps * SBS) {
                const int par = t_ >= A.g.Vh / 2 ? 1 : 0;
                const int i = colour_site(A.g, 1, t_ - par * (A.g.Vh / 2));
                Spinor<T> a, b;
                hop_site<P, false, SERIES_UNR>(A.g, MODE_CROSS, 0, par, i, z[1 - par], A.UP, a);
                load_spinor<P, false>(q[par], i, b);
                sp_axpy(a, kap, b);
                store_spinor<P>(A.fw2[par], i, a);
            }
            SAP_SYNC;
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Schwarz preconditioner over small 4-D blocks (SOLVER_SAPB)
//
// The same multiplicative cycle as sap_apply (all blocks of colour 0, then
// all blocks of colour 1 with the source corrected by the hops from the
// colour-0 blocks, each block solve the truncated geometric series of the
// even-odd reduced block operator), on blocks of bk[0] x .. x bk[3] sites
// (bk[mu] = 4 or 2, so a block starts on an even site and its local
// checkerboard is the global one).  A block's colour is the parity of the
// sum of its block coordinates.  One CTA solves one block at a time with
// the block's links and the vectors of its series in shared memory, so the
// series needs __syncthreads only; the system's barrier is met once per
// colour (2 per application instead of 4 nsap + 5).
// ---------------------------------------------------------------------------
constexpr int SAPB_BVH = SBS / 2;  // largest block: 2 SBS / 2 sites, 4^4

// shared-memory bytes of one CTA: links (rows 0-1 of U_mu(y), both
// parities) and three block vectors (odd source, even iterate, odd
// intermediate)
template <class T>
constexpr int sapb_smem_bytes()
{
    return (4 * 2 * 6 + 3 * 12) * SAPB_BVH * (int)sizeof(cx<T>);
}

// local coordinates of the block site with parity p and local eo index n
// (local lexicographic order with y3 fastest, as the lattice's)
__device__ __forceinline__ void blk_coords(const SolveArgs& A, int p, int n, int y[4])
{
    const int l = 2 * n;
    y[3] = l & (A.bk[3] - 1);
    int t = l >> A.lbk[3];
    y[2] = t & (A.bk[2] - 1);
    t >>= A.lbk[2];
    y[1] = t & (A.bk[1] - 1);
    y[0] = t >> A.lbk[1];
    y[3] += (y[0] + y[1] + y[2] + y[3] + p) & 1;
}

// block coordinates of the j-th block of colour c; false if the j-th block
// has the other colour (when nbk[3] is odd, all blocks are enumerated)
__device__ __forceinline__ bool blk_of(const SolveArgs& A, int c, int j, int B[4])
{
    int t = j;
    if ((A.nbk[3] & 1) == 0) {
        const int h3 = A.nbk[3] >> 1;
        const int b3 = t % h3;
        t /= h3;
        B[2] = t % A.nbk[2];
        t /= A.nbk[2];
        B[1] = t % A.nbk[1];
        B[0] = t / A.nbk[1];
        B[3] = 2 * b3 + ((B[0] + B[1] + B[2] + c) & 1);
        return true;
    }
    B[3] = t % A.nbk[3];
    t /= A.nbk[3];
    B[2] = t % A.nbk[2];
    t /= A.nbk[2];
    B[1] = t % A.nbk[1];
    B[0] = t / A.nbk[1];
    return ((B[0] + B[1] + B[2] + B[3]) & 1) == c;
}

// The hopping term inside one block (hops leaving the block dropped) at
// output site (pout, n), from the block vector `in` of parity 1 - pout in
// shared memory, computed by a pair of threads: thread s (0 or 1) projects
// spin row s of every neighbour, applies the link and accumulates output
// spins s (up) and 2 + s (lo).  The lower half of (1 + sg gamma_mu) psi
// mixes the two rows for mu = 1, 2; those parts belong to the partner's
// lower spin and are exchanged by one shuffle at the end.  Both threads of
// a pair take every branch together (the spin row is data, not control).
template <class T>
__device__ __forceinline__ void blk_hop_pair(const SolveArgs& A, const cx<T>* Ls, const cx<T>* in, int pout, int n,
                                             int s, bool on, cx<T> up[3], cx<T> lo[3])
{
    cx<T> ot[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) up[i] = lo[i] = ot[i] = mk(T(0), T(0));
    if (on) {
        const int bvh = A.bvh;
        int y[4];
        blk_coords(A, pout, n, y);
        const int l = ((y[0] * A.bk[1] + y[1]) * A.bk[2] + y[2]) * A.bk[3] + y[3];
        const T sig = s ? T(-1) : T(1);
        int stride = 1;
#pragma unroll
        for (int mu = 3; mu >= 0; --mu) {
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {  // forward, backward
                const bool inside = dir == 0 ? (y[mu] + 1 < A.bk[mu]) : (y[mu] > 0);
                if (inside) {
                    const int nn = (dir == 0 ? l + stride : l - stride) >> 1;
                    // forward: U_mu(y) at (pout, n); backward: U_mu(y - mu) at (1 - pout, nn)
                    const cx<T>* lp = Ls + (size_t)((mu * 2 + (dir == 0 ? pout : 1 - pout)) * 6) * bvh +
                                      (dir == 0 ? n : nn);
                    Su3<T> u;
#pragma unroll
                    for (int e = 0; e < 6; ++e) u.m[e / 3][e % 3] = lp[e * bvh];
                    complete_row2(u);
                    const int sg = dir == 0 ? -1 : +1;
                    // row s of the projection: h = p_s - sg a_s with a_s = p_(2+s)
                    // (mu 0), i p_(3-s) (mu 1), sig p_(3-s) (mu 2), sig i p_(2+s) (mu 3)
                    const int q = (mu == 0 || mu == 3) ? 2 + s : 3 - s;
                    cx<T> h[3];
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const cx<T> ps = in[(s * 3 + i) * bvh + nn];
                        const cx<T> pq = in[(q * 3 + i) * bvh + nn];
                        cx<T> a;
                        if (mu == 0) a = pq;
                        else if (mu == 1) a = mul_i(pq);
                        else if (mu == 2) a = sig * pq;
                        else a = sig * mul_i(pq);
                        h[i] = sg < 0 ? ps + a : ps - a;
                    }
                    cx<T> w[3];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
                        w[i] = dir == 0 ? u.m[i][0] * h[0] + u.m[i][1] * h[1] + u.m[i][2] * h[2]
                                        : cjmul(u.m[0][i], h[0]) + cjmul(u.m[1][i], h[1]) + cjmul(u.m[2][i], h[2]);
                    // upper spin s += w; lower spin 2 + t += sg l_t with l_t =
                    // -w_t (mu 0), i w_(1-t) (mu 1), sig_t w_(1-t) (mu 2), i sig_t w_t (mu 3)
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        up[i] = up[i] + w[i];
                        if (mu == 0) lo[i] = sg < 0 ? lo[i] + w[i] : lo[i] - w[i];
                        else if (mu == 3) lo[i] = lo[i] + (T)sg * sig * mul_i(w[i]);
                        else if (mu == 1) ot[i] = ot[i] + (T)sg * mul_i(w[i]);
                        else ot[i] = ot[i] - (T)sg * sig * w[i];
                    }
                }
            }
            stride *= A.bk[mu];
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        lo[i].re += __shfl_xor_sync(0xffffffffu, ot[i].re, 1);
        lo[i].im += __shfl_xor_sync(0xffffffffu, ot[i].im, 1);
    }
}

// z = K^-1 q with the 4-D block cycle above.  Full-lattice vectors in P;
// two system barriers.
template <int P>
__device__ bool sapb_apply(const SolveArgs& A, int sys, int cin, unsigned& epoch, const SpinorF* q, const SpinorF* z)
{
    typedef typename Real<P>::T T;
    extern __shared__ __align__(16) unsigned char sapb_dyn[];
    const int bvh = A.bvh;
    cx<T>* Ls = (cx<T>*)sapb_dyn;             // [4][2][6][bvh]
    cx<T>* so = Ls + 4 * 2 * 6 * SAPB_BVH;    // [12][bvh] odd source
    cx<T>* ev = so + 12 * SAPB_BVH;           // [12][bvh] even source, then iterate
    cx<T>* od = ev + 12 * SAPB_BVH;           // [12][bvh] odd intermediate
    const T kap = (T)A.kappa, k2 = (T)A.k2;
    const int tid = threadIdx.x;
    // pair mapping of the series phases: site n = tid / 2, spin row s = tid & 1
    const int pn = tid >> 1, ps = tid & 1;
    const bool pon = pn < bvh;
    const int nloop = (A.nbk[3] & 1) == 0 ? A.nblk / 2 : A.nblk;
    for (int c = 0; c < 2; ++c) {
        for (int j = cin; j < nloop; j += A.cps) {
            int B[4];
            if (!blk_of(A, c, j, B)) continue;  // uniform over the CTA
            // ---- links of the block and the source, one thread per site:
            // src = q, plus kappa times the hops from colour-0 blocks (c = 1)
            for (int t = tid; t < 2 * bvh; t += SBS) {
                const int p = t >= bvh ? 1 : 0, n = t - p * bvh;
                int y[4], x[4];
                blk_coords(A, p, n, y);
#pragma unroll
                for (int mu = 0; mu < 4; ++mu) x[mu] = B[mu] * A.bk[mu] + y[mu];
                const int lex = lex_of(A.g, x);
                const int gi = lex >> 1;
                Spinor<T> src, ext;
                load_spinor<P, false>(q[p], gi, src);
                sp_zero(ext);
                int stride = 1;
#pragma unroll
                for (int mu = 3; mu >= 0; --mu) {
                    Su3<T> u;
                    load_link<P>(A.UP, mu, p, gi, u);
#pragma unroll
                    for (int e = 0; e < 6; ++e) Ls[((mu * 2 + p) * 6 + e) * bvh + n] = u.m[e / 3][e % 3];
                    if (c == 1) {
                        // forward hop leaving the block
                        if (y[mu] == A.bk[mu] - 1) {
                            const int Bn = B[mu] + 1 == A.nbk[mu] ? 0 : B[mu] + 1;
                            if (((c - B[mu] + Bn) & 1) == 0) {
                                const bool wrap = x[mu] == A.g.L[mu] - 1;
                                const int nl = wrap ? lex + stride - A.g.L[mu] * stride : lex + stride;
                                Spinor<T> pz;
                                load_spinor<P, false>(z[1 - p], nl >> 1, pz);
                                HalfSp<T> hh, w;
                                project(mu, -1, pz, hh);
                                su3_mul_half(u, hh, w);
                                if (mu == 0 && wrap && A.g.bc_t < 0) {
#pragma unroll
                                    for (int a = 0; a < 2; ++a)
#pragma unroll
                                        for (int b = 0; b < 3; ++b) w.c[a][b] = -w.c[a][b];
                                }
                                accum_recon(mu, -1, w, ext);
                            }
                        }
                        // backward hop leaving the block
                        if (y[mu] == 0) {
                            const int Bn = B[mu] == 0 ? A.nbk[mu] - 1 : B[mu] - 1;
                            if (((c - B[mu] + Bn) & 1) == 0) {
                                const bool wrap = x[mu] == 0;
                                const int nl = wrap ? lex - stride + A.g.L[mu] * stride : lex - stride;
                                Spinor<T> pz;
                                load_spinor<P, false>(z[1 - p], nl >> 1, pz);
                                Su3<T> ub;
                                load_link<P>(A.UP, mu, 1 - p, nl >> 1, ub);
                                HalfSp<T> hh, w;
                                project(mu, +1, pz, hh);
                                su3_dagmul_half(ub, hh, w);
                                if (mu == 0 && wrap && A.g.bc_t < 0) {
#pragma unroll
                                    for (int a = 0; a < 2; ++a)
#pragma unroll
                                        for (int b = 0; b < 3; ++b) w.c[a][b] = -w.c[a][b];
                                }
                                accum_recon(mu, +1, w, ext);
                            }
                        }
                    }
                    stride *= A.g.L[mu];
                }
                if (c == 1) sp_axpy(ext, kap, src);  // ext <- src + kappa ext
                else ext = src;
                cx<T>* dst = p ? so : ev;
#pragma unroll
                for (int k = 0; k < 12; ++k) dst[k * bvh + n] = ext.c[k / 3][k % 3];
            }
            __syncthreads();
            // ---- be = src_e + kappa H_eo src_o (the pair's two spins kept
            // in registers); the series starts from u_0 = be
            cx<T> be[2][3];
            {
                cx<T> up[3], lo[3];
                blk_hop_pair<T>(A, Ls, so, 0, pn, ps, pon, up, lo);
                if (pon) {
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        be[0][i] = ev[(ps * 3 + i) * bvh + pn] + kap * up[i];
                        be[1][i] = ev[((2 + ps) * 3 + i) * bvh + pn] + kap * lo[i];
                        ev[(ps * 3 + i) * bvh + pn] = be[0][i];
                        ev[((2 + ps) * 3 + i) * bvh + pn] = be[1][i];
                    }
                }
            }
            __syncthreads();
            // ---- u <- be + kappa^2 H_eo H_oe u, nsap times
            for (int it = 0; it < A.nsap; ++it) {
                cx<T> up[3], lo[3];
                blk_hop_pair<T>(A, Ls, ev, 1, pn, ps, pon, up, lo);
                if (pon) {
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        od[(ps * 3 + i) * bvh + pn] = up[i];
                        od[((2 + ps) * 3 + i) * bvh + pn] = lo[i];
                    }
                }
                __syncthreads();
                blk_hop_pair<T>(A, Ls, od, 0, pn, ps, pon, up, lo);
                if (pon) {
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        ev[(ps * 3 + i) * bvh + pn] = be[0][i] + k2 * up[i];
                        ev[((2 + ps) * 3 + i) * bvh + pn] = be[1][i] + k2 * lo[i];
                    }
                }
                __syncthreads();
            }
            // ---- y_o = src_o + kappa H_oe u (into the odd intermediate)
            {
                cx<T> up[3], lo[3];
                blk_hop_pair<T>(A, Ls, ev, 1, pn, ps, pon, up, lo);
                if (pon) {
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        od[(ps * 3 + i) * bvh + pn] = so[(ps * 3 + i) * bvh + pn] + kap * up[i];
                        od[((2 + ps) * 3 + i) * bvh + pn] = so[((2 + ps) * 3 + i) * bvh + pn] + kap * lo[i];
                    }
                }
            }
            __syncthreads();
            // ---- z on the block (y_e = u, y_o), one thread per site
            for (int t = tid; t < 2 * bvh; t += SBS) {
                const int p = t >= bvh ? 1 : 0, n = t - p * bvh;
                int y[4], x[4];
                blk_coords(A, p, n, y);
#pragma unroll
                for (int mu = 0; mu < 4; ++mu) x[mu] = B[mu] * A.bk[mu] + y[mu];
                const cx<T>* srcv = p ? od : ev;
                Spinor<T> out;
#pragma unroll
                for (int k = 0; k < 12; ++k) out.c[k / 3][k % 3] = srcv[k * bvh + n];
                store_spinor<P>(z[p], lex_of(A.g, x) >> 1, out);
            }
            __syncthreads();
        }
        SAP_SYNC;
    }
    return true;
}

#define FOR_FULL_SITES \
    for (int t_ = cin * SBS + (int)threadIdx.x; t_ < 2 * A.g.Vh; t_ += A.cps * SBS)

// Schwarz-preconditioned BiCGstab (right preconditioning, K^-1 = sap_apply)
// on the full lattice for M y = (r64 / |r64|, 0) in P: M y = (r, 0) makes
// y_e the solution of the even-odd reduced system (1 - kappa^2 H_eo H_oe)
// y_e = r, so the caller's double defect correction on that system is
// unchanged (fy[0] is the caller's e).  Returns false when a barrier wait
// gave up.
template <int P>
__device__ bool sap_bicgstab(const SolveArgs& A, int sys, int cin, unsigned& epoch, SysSt& S, double* red, int& rb)
{
    typedef typename Real<P>::T T;
    constexpr int PE = (P == PREC64) ? PREC64 : PREC32;
    typedef typename Real<PE>::T TE;
    const int tid = threadIdx.x;
    const T kap = (T)A.kappa;
    // ---- start: r = rh = p = (r64 / |r64|, 0), y = 0
    {
        double q = 0.0;
        if (S.active) {
            const double sc = 1.0 / sqrt(S.rn2);
            FOR_FULL_SITES
            {
                const int par = t_ >= A.g.Vh ? 1 : 0, i = t_ - par * A.g.Vh;
                Spinor<T> r;
                Spinor<TE> z;
                sp_zero(z);
                sp_zero(r);
                if (par == 0) {
                    Spinor<double> r6;
                    load_spinor<PREC64, false>(A.r64, i, r6);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) r.c[s][c] = mk((T)(sc * r6.c[s][c].re), (T)(sc * r6.c[s][c].im));
                }
                store_spinor<P>(A.fr[par], i, r);
                load_spinor<P, false>(A.fr[par], i, r);  // the stored (rounded) vector
                store_spinor<P>(A.frh[par], i, r);
                store_spinor<P>(A.fp[par], i, r);
                store_spinor<PE>(A.fy[par], i, z);
                q += nrm_acc(r);
            }
        }
        reduce_put(A, q, 0.0, 0.0, 1, rb);
        SAP_SYNC;
        gather_own(A, sys, 1, red, rb);
        if (tid == 0) {
            S.rho = make_double2(red[0], 0.0);
            S.idone = !S.active;
            S.itc = 0;
            const double need = 0.5 * A.tol * sqrt(S.bn2 / fmax(S.rn2, 1e-300));
            const double it = fmax(A.inner_tol, need);
            S.itol2 = it * it;
        }
        __syncthreads();
    }
    for (;;) {
        if (S.idone) break;
        // zp = K^-1 p ; v = M zp ; <rh, v>
        if (!(A.method == SOLVER_SAPB ? sapb_apply<P>(A, sys, cin, epoch, A.fp, A.fzp)
                                      : sap_apply<P>(A, sys, cin, epoch, A.fp, A.fzp)))
            return false;
        {
            double qr = 0.0, qi = 0.0;
            FOR_FULL_SITES
            {
                const int par = t_ >= A.g.Vh ? 1 : 0, i = t_ - par * A.g.Vh;
                Spinor<T> a, z, rh;
                hop_site<P, false, SERIES_UNR>(A.g, MODE_ALL, 0, par, i, A.fzp[1 - par], A.UP, a);
                load_spinor<P, false>(A.fzp[par], i, z);
                sp_axpy(a, -kap, z);
                store_spinor<P>(A.fv[par], i, a);
                if (P == PREC16 || P == PRECBF) load_spinor<P, false>(A.fv[par], i, a);
                load_spinor<P, false>(A.frh[par], i, rh);
                cdot_acc(rh, a, qr, qi);
            }
            reduce_put(A, qr, qi, 0.0, 2, rb);
            SAP_SYNC;
            gather_own(A, sys, 2, red, rb);
            if (tid == 0) {
                const double2 d = make_double2(red[0], red[1]);
                const double2 al = cdiv(S.rho, d);
                if (!finite2(al) || (d.x == 0.0 && d.y == 0.0)) {
                    S.idone = 1;
                    S.alpha = make_double2(0.0, 0.0);
                } else {
                    S.alpha = al;
                }
            }
            __syncthreads();
        }
        if (S.idone) break;
        // s = r - alpha v
        {
            const cx<T> al = mk((T)S.alpha.x, (T)S.alpha.y);
            FOR_FULL_SITES
            {
                const int par = t_ >= A.g.Vh ? 1 : 0, i = t_ - par * A.g.Vh;
                Spinor<T> r, v;
                load_spinor<P, false>(A.fr[par], i, r);
                load_spinor<P, false>(A.fv[par], i, v);
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) r.c[s][c] = r.c[s][c] - al * v.c[s][c];
                store_spinor<P>(A.fs[par], i, r);
            }
            SAP_SYNC;
        }
        // zs = K^-1 s ; t = M zs ; <t, s>, <t, t>
        if (!(A.method == SOLVER_SAPB ? sapb_apply<P>(A, sys, cin, epoch, A.fs, A.fzs)
                                      : sap_apply<P>(A, sys, cin, epoch, A.fs, A.fzs)))
            return false;
        {
            double qr = 0.0, qi = 0.0, qt = 0.0;
            FOR_FULL_SITES
            {
                const int par = t_ >= A.g.Vh ? 1 : 0, i = t_ - par * A.g.Vh;
                Spinor<T> a, z, ss;
                hop_site<P, false, SERIES_UNR>(A.g, MODE_ALL, 0, par, i, A.fzs[1 - par], A.UP, a);
                load_spinor<P, false>(A.fzs[par], i, z);
                sp_axpy(a, -kap, z);
                store_spinor<P>(A.ft[par], i, a);
                if (P == PREC16 || P == PRECBF) load_spinor<P, false>(A.ft[par], i, a);
                load_spinor<P, false>(A.fs[par], i, ss);
                cdot_acc(a, ss, qr, qi);
                qt += nrm_acc(a);
            }
            reduce_put(A, qr, qi, qt, 3, rb);
            SAP_SYNC;
            gather_own(A, sys, 3, red, rb);
            if (tid == 0) {
                const double tt = red[2];
                const double2 om = make_double2(red[0] / tt, red[1] / tt);
                if (!(tt > 0.0) || !finite2(om)) {
                    S.omega = make_double2(0.0, 0.0);
                    S.idone = 2;  // keep alpha zp, stop afterwards
                } else {
                    S.omega = om;
                }
            }
            __syncthreads();
        }
        // y += alpha zp + omega zs ; r = s - omega t ; <rh, r>, |r|^2
        {
            double qr = 0.0, qi = 0.0, qn = 0.0;
            const cx<T> al = mk((T)S.alpha.x, (T)S.alpha.y);
            const cx<T> om = mk((T)S.omega.x, (T)S.omega.y);
            FOR_FULL_SITES
            {
                const int par = t_ >= A.g.Vh ? 1 : 0, i = t_ - par * A.g.Vh;
                Spinor<T> zp, zs, ss, tt, rh;
                Spinor<TE> yy;
                load_spinor<PE, false>(A.fy[par], i, yy);
                load_spinor<P, false>(A.fzp[par], i, zp);
                load_spinor<P, false>(A.fzs[par], i, zs);
                load_spinor<P, false>(A.fs[par], i, ss);
                load_spinor<P, false>(A.ft[par], i, tt);
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const cx<T> d = al * zp.c[s][c] + om * zs.c[s][c];
                        yy.c[s][c] = yy.c[s][c] + mk((TE)d.re, (TE)d.im);
                        ss.c[s][c] = ss.c[s][c] - om * tt.c[s][c];
                    }
                store_spinor<PE>(A.fy[par], i, yy);
                store_spinor<P>(A.fr[par], i, ss);
                if (P == PREC16 || P == PRECBF) load_spinor<P, false>(A.fr[par], i, ss);
                load_spinor<P, false>(A.frh[par], i, rh);
                cdot_acc(rh, ss, qr, qi);
                qn += nrm_acc(ss);
            }
            reduce_put(A, qr, qi, qn, 3, rb);
            SAP_SYNC;
            gather_own(A, sys, 3, red, rb);
            if (tid == 0) {
                S.it += 1;
                S.itc += 1;
                const double2 rn = make_double2(red[0], red[1]);
                S.rr = red[2];
                if (S.idone == 2 || S.itc >= A.max_inner || S.it >= A.max_iter || !(S.rr > S.itol2) ||
                    !finite2(rn) || S.rr > 1e8) {
                    S.idone = 1;
                } else {
                    S.beta = cmul(cdiv(rn, S.rho), cdiv(S.alpha, S.omega));
                    if (!finite2(S.beta)) S.idone = 1;
                    S.rho = rn;
                }
            }
            if (tid == 0 && S.idone) S.idone = 1;
            __syncthreads();
        }
        if (S.idone) break;
        // p = r + beta (p - omega v)
        {
            const cx<T> be = mk((T)S.beta.x, (T)S.beta.y);
            const cx<T> om = mk((T)S.omega.x, (T)S.omega.y);
            FOR_FULL_SITES
            {
                const int par = t_ >= A.g.Vh ? 1 : 0, i = t_ - par * A.g.Vh;
                Spinor<T> r, pp, v;
                load_spinor<P, false>(A.fr[par], i, r);
                load_spinor<P, false>(A.fp[par], i, pp);
                load_spinor<P, false>(A.fv[par], i, v);
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) r.c[s][c] = r.c[s][c] + be * (pp.c[s][c] - om * v.c[s][c]);
                store_spinor<P>(A.fp[par], i, r);
            }
            SAP_SYNC;
        }
    }
    SAP_SYNC;
    return true;
}

#undef SAP_SYNC
#undef FOR_COLOUR_SITES
#undef FOR_FULL_SITES

template <int P, bool SAP>
__global__ void __launch_bounds__(SBS, P == PREC64 ? 1 : 2) k_solve(SolveArgs A)
{
    typedef typename Real<P>::T T;
    constexpr int PE = (P == PREC64) ? PREC64 : PREC32;
    typedef typename Real<PE>::T TE;
    // the double residual sweeps: FP64 for a double solve, double-float
    // arithmetic on the double fields and links for a mixed one
    constexpr int PR = (P == PREC64) ? PREC64 : PRECDF;
    typedef typename Real<PR>::T TR;
    // t64 = H_oe x between the two residual sweeps: kept as df pairs in the
    // mixed case (no conversion to double and back)
    constexpr int PT = (P == PREC64) ? PREC64 : PRECDS;
    constexpr bool WORDS = (P == PREC32);
    const int cta = blockIdx.x, tid = threadIdx.x;
    const int sys = cta / A.cps, cin = cta - sys * A.cps;
    const bool leader = (cin == 0 && tid == 0);  // writes the system's results
    const int base = (A.mode == MODE_INTRA) ? (A.slab0 + sys * A.slabstep) * A.g.Sh : 0;
    __shared__ SysSt S;
    __shared__ double red[NQ];
    unsigned epoch = 0;
    int rb = 0;  // partial-sum buffer

    // ---- x = 0, r64 = b, |b|^2; with an initial guess (x given): |b|^2 and
    // t64 = H_oe x here, r64 = b - diag x + k2 H_eo t64 below
    {
        double q = 0.0;
        FOR_SITES
        {
            const int i = base + j_;
            Spinor<double> bb, z;
            load_spinor<PREC64, true>(A.b, i, bb);
            if (A.guess) {
                Spinor<TR> hz;
                hop_site<PR, false, SOLVE_UNR>(A.g, A.mode, 0, 1, i, A.x, A.U64, hz);
                store_spinor<PT>(A.t64, i, hz);
            } else {
                store_spinor<PREC64>(A.r64, i, bb);
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) z.c[s][c] = mk(0.0, 0.0);
                store_spinor<PREC64>(A.x, i, z);
            }
            q += nrm_acc(bb);
        }
        reduce_put(A, q, 0.0, 0.0, 1, rb);
        SYNC_OR_RETURN;
        gather_own(A, sys, 1, red, rb);
        if (tid == 0) {
            S.bn2 = red[0];
            S.rn2 = red[0];
            S.it = 0;
        }
        __syncthreads();
    }
    if (A.guess) {
        double q = 0.0;
        FOR_SITES
        {
            const int i = base + j_;
            Spinor<double> a, xx, bb;
            {
                Spinor<TR> ha;
                hop_site<PT, false, SOLVE_UNR>(A.g, A.mode, 0, 0, i, A.t64, A.U64, ha);
                to_double(ha, a);
            }
            load_spinor<PREC64, false>(A.x, i, xx);
            load_spinor<PREC64, true>(A.b, i, bb);
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) a.c[s][c] = bb.c[s][c] - A.diag * xx.c[s][c] + A.k2 * a.c[s][c];
            store_spinor<PREC64>(A.r64, i, a);
            q += nrm_acc(a);
        }
        reduce_put(A, q, 0.0, 0.0, 1, rb);
        SYNC_OR_RETURN;
        gather_own(A, sys, 1, red, rb);
        if (tid == 0) S.rn2 = red[0];
        __syncthreads();
        if (!(S.bn2 > 0.0)) FOR_SITES  // b = 0: the solution is 0, whatever the guess
            {
                Spinor<double> z;
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) z.c[s][c] = mk(0.0, 0.0);
                store_spinor<PREC64>(A.x, base + j_, z);
            }
    }

    int outer = 0, final_flag = F_DONE;
    for (;;) {
        // the system's state: every CTA of the system takes the same decision
        // from the same gathered sums
        if (tid == 0) {
            const bool nan = !isfinite(S.rn2);
            const bool conv = !(S.rn2 > A.tol * A.tol * S.bn2) || !(S.bn2 > 0.0);
            S.active = (!nan && !conv) ? 1 : 0;
            int f = nan ? F_NAN : conv ? F_DONE : F_ACTIVE;
            if (f == F_ACTIVE && (outer >= A.max_outer || S.it >= A.max_iter)) f = F_MAXIT;
            S.flag = f;
        }
        __syncthreads();
        if (S.flag != F_ACTIVE) {
            final_flag = S.flag;
            break;
        }
        ++outer;

        if constexpr (SAP) {
            if (!sap_bicgstab<P>(A, sys, cin, epoch, S, red, rb)) return;
        } else {
        // ---- inner start: r = rh = p = r64 / |r64|, e = 0
        {
            double q = 0.0;
            if (S.active && WORDS) {
                const double sc = 1.0 / sqrt(S.rn2);
                const double2* r6 = (const double2*)A.r64.v;
                float qf = 0.f;
                FOR_WORDS
                {
                    const int k = f_ / A.nsite, i = base + (f_ % A.nsite);
                    const size_t a = (size_t)k * A.g.Vh + i;
                    const double2 d0 = r6[(size_t)(2 * k) * A.g.Vh + i], d1 = r6[(size_t)(2 * k + 1) * A.g.Vh + i];
                    const float4 w = make_float4((float)(sc * d0.x), (float)(sc * d0.y), (float)(sc * d1.x),
                                                 (float)(sc * d1.y));
                    W4(A.r)[a] = w;
                    W4(A.rh)[a] = w;
                    W4(A.p)[a] = w;
                    W4(A.e)[a] = make_float4(0.f, 0.f, 0.f, 0.f);
                    qf += nrm2w(w);
                }
                q = qf;
            } else if (S.active) {
                const double sc = 1.0 / sqrt(S.rn2);
                FOR_SITES
                {
                    const int i = base + j_;
                    Spinor<double> r6;
                    load_spinor<PREC64, false>(A.r64, i, r6);
                    Spinor<T> r;
                    Spinor<TE> z;
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            r.c[s][c] = mk((T)(sc * r6.c[s][c].re), (T)(sc * r6.c[s][c].im));
                            z.c[s][c] = mk((TE)0, (TE)0);
                        }
                    store_spinor<P>(A.r, i, r);
                    load_spinor<P, false>(A.r, i, r);  // the stored (rounded) vector
                    store_spinor<P>(A.rh, i, r);
                    store_spinor<P>(A.p, i, r);
                    store_spinor<PE>(A.e, i, z);
                    q += nrm_acc(r);
                }
            }
            reduce_put(A, q, 0.0, 0.0, 1, rb);
            SYNC_OR_RETURN;
            gather_own(A, sys, 1, red, rb);
            if (tid == 0) {
                S.rho = make_double2(red[0], 0.0);
                S.idone = !S.active;
                S.itc = 0;
                const double need = 0.5 * A.tol * sqrt(S.bn2 / fmax(S.rn2, 1e-300));
                const double it = fmax(A.inner_tol, need);
                S.itol2 = it * it;
            }
            __syncthreads();
        }

        if (A.method == SOLVER_SERIES) {
            // ---- geometric series (Sec. 3, the solver of the block terms):
            // p <- (r + k2 H_eo H_oe p) / diag from p = r; before an update
            // the inner residual is r - A p = diag (p_new - p).  Two
            // barriers per iteration; the residual is reduced every second
            // iteration only (and at the iteration limits), which costs at
            // most one extra iteration per inner solve.
            const T k2 = (T)A.k2, dinv = (T)(1.0 / A.diag);
            for (;;) {
                if (S.idone) break;
                const bool chk = (S.itc & 1) || S.itc + 1 >= A.max_inner || S.it + 1 >= A.max_iter;
                FOR_SITES
                {
                    const int i = base + j_;
                    Spinor<T> a;
                    hop_site<P, false, SERIES_UNR>(A.g, A.mode, 0, 1, i, A.p, A.UP, a);
                    store_spinor<P>(A.tmp, i, a);
                }
                SYNC_OR_RETURN;
                double q = 0.0;
                FOR_SITES
                    {
                        const int i = base + j_;
                        Spinor<T> a, pp, rr;
                        hop_site<P, false, SERIES_UNR>(A.g, A.mode, 0, 0, i, A.tmp, A.UP, a);
                        load_spinor<P, false>(A.p, i, pp);
                        load_spinor<P, false>(A.r, i, rr);
#pragma unroll
                        for (int s = 0; s < 4; ++s)
#pragma unroll
                            for (int c = 0; c < 3; ++c) a.c[s][c] = dinv * (rr.c[s][c] + k2 * a.c[s][c]);
                        store_spinor<P>(A.p, i, a);
                        if (chk) {
                            if (P == PREC16 || P == PRECBF) load_spinor<P, false>(A.p, i, a);
#pragma unroll
                            for (int s = 0; s < 4; ++s)
#pragma unroll
                                for (int c = 0; c < 3; ++c) pp.c[s][c] = a.c[s][c] - pp.c[s][c];
                            q += nrm_acc(pp);
                        }
                    }
                if (!chk) {
                    SYNC_OR_RETURN;
                    if (tid == 0) {
                        S.it += 1;
                        S.itc += 1;
                    }
                    __syncthreads();
                    continue;
                }
                reduce_put(A, q, 0.0, 0.0, 1, rb);
                SYNC_OR_RETURN;
                gather_own(A, sys, 1, red, rb);
                if (tid == 0) {
                    S.it += 1;
                    S.itc += 1;
                    const double res2 = A.diag * A.diag * red[0];
                    if (!(res2 > S.itol2) || S.itc >= A.max_inner || S.it >= A.max_iter) S.idone = 1;
                    // a series that grows (spectral radius above one) cannot
                    // converge: report the system as not converged
                    if (!isfinite(res2) || (S.itc >= 16 && res2 > 1e6)) {
                        S.idone = 1;
                        S.it = A.max_iter;
                    }
                }
                __syncthreads();
            }
            // e = p
            if (S.active) FOR_SITES
                {
                    const int i = base + j_;
                    Spinor<T> pp;
                    Spinor<TE> ee;
                    load_spinor<P, false>(A.p, i, pp);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) ee.c[s][c] = mk((TE)pp.c[s][c].re, (TE)pp.c[s][c].im);
                    store_spinor<PE>(A.e, i, ee);
                }
            SYNC_OR_RETURN;
        } else {
        if constexpr (P == PREC32) {
            // ---- BiCGstab with the vector updates folded into the hopping
            // phases: s = r - alpha v is formed where H_oe s reads it (at the
            // neighbours) and where the next phase keeps it; the update
            // p = r + beta (p - omega v) waits for the next iteration, whose
            // H_oe p forms it at the neighbours and whose second phase keeps
            // it.  Five barriers per iteration (seven unfolded); the same
            // word-wise single-precision operations as the unfolded form.
            bool pend = false;  // p = r + beta (p - omega v) not yet formed
            const T k2 = (T)A.k2, dg = (T)A.diag;
            for (;;) {
                if (S.idone) break;
                const float2 pbe = make_float2((float)S.beta.x, (float)S.beta.y);
                const float2 pmom = make_float2(-(float)S.omega.x, -(float)S.omega.y);
                // tmp = H_oe p'
                if (pend) {
                    FOR_SITES
                    {
                        const int i = base + j_;
                        Spinor<T> a;
                        hop_site_ld<P, SOLVE_UNR>(A.g, A.mode, 0, 1, i,
                                       [&](int j, Spinor<T>& sp) { load_axpypz32(A.v, A.p, A.r, pmom, pbe, j, sp); },
                                       A.UP, a);
                        store_spinor<P>(A.tmp, i, a);
                    }
                } else {
                    FOR_SITES
                    {
                        const int i = base + j_;
                        Spinor<T> a;
                        hop_site<P, false, SOLVE_UNR>(A.g, A.mode, 0, 1, i, A.p, A.UP, a);
                        store_spinor<P>(A.tmp, i, a);
                    }
                }
                SYNC_OR_RETURN;
                // p = p' ; v = dg p - k2 H_eo tmp ; <rh, v>
                {
                    double qr = 0.0, qi = 0.0;
                    FOR_SITES
                    {
                        const int i = base + j_;
                        Spinor<T> a, pp, rh;
                        hop_site<P, false, SOLVE_UNR>(A.g, A.mode, 0, 0, i, A.tmp, A.UP, a);
                        if (pend) {
                            load_axpypz32(A.v, A.p, A.r, pmom, pbe, i, pp);
                            store_spinor<P>(A.p, i, pp);
                        } else {
                            load_spinor<P, false>(A.p, i, pp);
                        }
#pragma unroll
                        for (int s = 0; s < 4; ++s)
#pragma unroll
                            for (int c = 0; c < 3; ++c) a.c[s][c] = dg * pp.c[s][c] - k2 * a.c[s][c];
                        store_spinor<P>(A.v, i, a);
                        load_spinor<P, false>(A.rh, i, rh);
                        cdot_acc(rh, a, qr, qi);
                    }
                    reduce_put(A, qr, qi, 0.0, 2, rb);
                    SYNC_OR_RETURN;
                    gather_own(A, sys, 2, red, rb);
                    if (tid == 0) {
                        const double2 d = make_double2(red[0], red[1]);
                        const double2 al = cdiv(S.rho, d);
                        if (!finite2(al) || (d.x == 0.0 && d.y == 0.0)) {
                            S.idone = 1;
                            S.alpha = make_double2(0.0, 0.0);
                        } else {
                            S.alpha = al;
                        }
                    }
                    __syncthreads();
                }
                pend = false;
                if (S.idone) break;
                const float2 mal = make_float2(-(float)S.alpha.x, -(float)S.alpha.y);
                // tmp = H_oe s, s = r - alpha v formed at the neighbours
                FOR_SITES
                {
                    const int i = base + j_;
                    Spinor<T> a;
                    hop_site_ld<P, SOLVE_UNR>(A.g, A.mode, 0, 1, i,
                                   [&](int j, Spinor<T>& sp) { load_axpy32(A.v, A.r, mal, j, sp); }, A.UP, a);
                    store_spinor<P>(A.tmp, i, a);
                }
                SYNC_OR_RETURN;
                // s = r - alpha v (kept) ; t = dg s - k2 H_eo tmp ; <t, s>, <t, t>
                {
                    double qr = 0.0, qi = 0.0, qt = 0.0;
                    FOR_SITES
                    {
                        const int i = base + j_;
                        Spinor<T> a, ss;
                        hop_site<P, false, SOLVE_UNR>(A.g, A.mode, 0, 0, i, A.tmp, A.UP, a);
                        load_axpy32(A.v, A.r, mal, i, ss);
                        store_spinor<P>(A.s, i, ss);
#pragma unroll
                        for (int s = 0; s < 4; ++s)
#pragma unroll
                            for (int c = 0; c < 3; ++c) a.c[s][c] = dg * ss.c[s][c] - k2 * a.c[s][c];
                        store_spinor<P>(A.t, i, a);
                        cdot_acc(a, ss, qr, qi);
                        qt += nrm_acc(a);
                    }
                    reduce_put(A, qr, qi, qt, 3, rb);
                    SYNC_OR_RETURN;
                    gather_own(A, sys, 3, red, rb);
                    if (tid == 0) {
                        const double tt = red[2];
                        const double2 om = make_double2(red[0] / tt, red[1] / tt);
                        if (!(tt > 0.0) || !finite2(om)) {
                            S.omega = make_double2(0.0, 0.0);
                            S.idone = 2;  // keep alpha p, stop afterwards
                        } else {
                            S.omega = om;
                        }
                    }
                    __syncthreads();
                }
                // e += alpha p + omega s ; r = s - omega t ; <rh, r>, |r|^2
                {
                    double qr = 0.0, qi = 0.0, qn = 0.0;
                    const float2 al = make_float2((float)S.alpha.x, (float)S.alpha.y);
                    const float2 om = make_float2((float)S.omega.x, (float)S.omega.y);
                    const float2 mom = make_float2(-om.x, -om.y);
                    float fr = 0.f, fi = 0.f, fn = 0.f;
                    FOR_WORDS
                    {
                        WORD_ADDR;
                        const float4 ss = W4(A.s)[a];
                        W4(A.e)[a] = caxpy2(om, ss, caxpy2(al, W4(A.p)[a], W4(A.e)[a]));
                        const float4 rr = caxpy2(mom, W4(A.t)[a], ss);
                        W4(A.r)[a] = rr;
                        cdot2(W4(A.rh)[a], rr, fr, fi);
                        fn += nrm2w(rr);
                    }
                    qr = fr;
                    qi = fi;
                    qn = fn;
                    reduce_put(A, qr, qi, qn, 3, rb);
                    SYNC_OR_RETURN;
                    gather_own(A, sys, 3, red, rb);
                    if (tid == 0) {
                        S.it += 1;
                        S.itc += 1;
                        const double2 rn = make_double2(red[0], red[1]);
                        S.rr = red[2];
                        if (S.idone == 2 || S.itc >= A.max_inner || S.it >= A.max_iter || !(S.rr > S.itol2) ||
                            !finite2(rn) || S.rr > 1e8) {
                            S.idone = 1;
                        } else {
                            S.beta = cmul(cdiv(rn, S.rho), cdiv(S.alpha, S.omega));
                            if (!finite2(S.beta)) S.idone = 1;
                            S.rho = rn;
                        }
                    }
                    if (tid == 0 && S.idone) S.idone = 1;
                    __syncthreads();
                }
                pend = !S.idone;
            }
        } else
        // ---- BiCGstab: seven barriers per iteration
        for (;;) {
            if (S.idone) break;
            const bool act = true;
            // tmp = H_oe p
            FOR_SITES
            {
                const int i = base + j_;
                Spinor<T> a;
                hop_site<P, false, SOLVE_UNR>(A.g, A.mode, 0, 1, i, A.p, A.UP, a);
                store_spinor<P>(A.tmp, i, a);
            }
            SYNC_OR_RETURN;
            // v = p - k2 H_eo tmp ; <rh, v>
            {
                double qr = 0.0, qi = 0.0;
                if (act) {
                    const T k2 = (T)A.k2, dg = (T)A.diag;
                    FOR_SITES
                    {
                        const int i = base + j_;
                        Spinor<T> a, pp, rh;
                        hop_site<P, false, SOLVE_UNR>(A.g, A.mode, 0, 0, i, A.tmp, A.UP, a);
                        load_spinor<P, false>(A.p, i, pp);
#pragma unroll
                        for (int s = 0; s < 4; ++s)
#pragma unroll
                            for (int c = 0; c < 3; ++c) a.c[s][c] = dg * pp.c[s][c] - k2 * a.c[s][c];
                        store_spinor<P>(A.v, i, a);
                        if (P == PREC16 || P == PRECBF) load_spinor<P, false>(A.v, i, a);
                        load_spinor<P, false>(A.rh, i, rh);
                        cdot_acc(rh, a, qr, qi);
                    }
                }
                reduce_put(A, qr, qi, 0.0, 2, rb);
                SYNC_OR_RETURN;
                gather_own(A, sys, 2, red, rb);
                if (tid == 0 && act) {
                    const double2 d = make_double2(red[0], red[1]);
                    const double2 al = cdiv(S.rho, d);
                    if (!finite2(al) || (d.x == 0.0 && d.y == 0.0)) {
                        S.idone = 1;
                        S.alpha = make_double2(0.0, 0.0);
                    } else {
                        S.alpha = al;
                    }
                }
                __syncthreads();
            }
            const bool act2 = act && !S.idone;
            // s = r - alpha v
            if (act2 && WORDS) {
                const float2 al = make_float2(-(float)S.alpha.x, -(float)S.alpha.y);
                FOR_WORDS
                {
                    WORD_ADDR;
                    W4(A.s)[a] = caxpy2(al, W4(A.v)[a], W4(A.r)[a]);
                }
            } else if (act2) {
                const cx<T> al = mk((T)S.alpha.x, (T)S.alpha.y);
                FOR_SITES
                {
                    const int i = base + j_;
                    Spinor<T> r, v;
                    load_spinor<P, false>(A.r, i, r);
                    load_spinor<P, false>(A.v, i, v);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) r.c[s][c] = r.c[s][c] - al * v.c[s][c];
                    store_spinor<P>(A.s, i, r);
                }
            }
            SYNC_OR_RETURN;
            // tmp = H_oe s
            if (act2) FOR_SITES
                {
                    const int i = base + j_;
                    Spinor<T> a;
                    hop_site<P, false, SOLVE_UNR>(A.g, A.mode, 0, 1, i, A.s, A.UP, a);
                    store_spinor<P>(A.tmp, i, a);
                }
            SYNC_OR_RETURN;
            // t = s - k2 H_eo tmp ; <t, s>, <t, t>
            {
                double qr = 0.0, qi = 0.0, qt = 0.0;
                if (act2) {
                    const T k2 = (T)A.k2, dg = (T)A.diag;
                    FOR_SITES
                    {
                        const int i = base + j_;
                        Spinor<T> a, ss;
                        hop_site<P, false, SOLVE_UNR>(A.g, A.mode, 0, 0, i, A.tmp, A.UP, a);
                        load_spinor<P, false>(A.s, i, ss);
#pragma unroll
                        for (int s = 0; s < 4; ++s)
#pragma unroll
                            for (int c = 0; c < 3; ++c) a.c[s][c] = dg * ss.c[s][c] - k2 * a.c[s][c];
                        store_spinor<P>(A.t, i, a);
                        if (P == PREC16 || P == PRECBF) load_spinor<P, false>(A.t, i, a);
                        cdot_acc(a, ss, qr, qi);
                        qt += nrm_acc(a);
                    }
                }
                reduce_put(A, qr, qi, qt, 3, rb);
                SYNC_OR_RETURN;
                gather_own(A, sys, 3, red, rb);
                if (tid == 0 && act2) {
                    const double tt = red[2];
                    const double2 om = make_double2(red[0] / tt, red[1] / tt);
                    if (!(tt > 0.0) || !finite2(om)) {
                        S.omega = make_double2(0.0, 0.0);
                        S.idone = 2;  // keep alpha p, stop afterwards
                    } else {
                        S.omega = om;
                    }
                }
                __syncthreads();
            }
            // e += alpha p + omega s ; r = s - omega t ; <rh, r>, |r|^2
            {
                double qr = 0.0, qi = 0.0, qn = 0.0;
                if (act2 && WORDS) {
                    const float2 al = make_float2((float)S.alpha.x, (float)S.alpha.y);
                    const float2 om = make_float2((float)S.omega.x, (float)S.omega.y);
                    const float2 mom = make_float2(-om.x, -om.y);
                    float fr = 0.f, fi = 0.f, fn = 0.f;
                    FOR_WORDS
                    {
                        WORD_ADDR;
                        const float4 ss = W4(A.s)[a];
                        W4(A.e)[a] = caxpy2(om, ss, caxpy2(al, W4(A.p)[a], W4(A.e)[a]));
                        const float4 rr = caxpy2(mom, W4(A.t)[a], ss);
                        W4(A.r)[a] = rr;
                        cdot2(W4(A.rh)[a], rr, fr, fi);
                        fn += nrm2w(rr);
                    }
                    qr = fr;
                    qi = fi;
                    qn = fn;
                } else if (act2) {
                    const cx<T> al = mk((T)S.alpha.x, (T)S.alpha.y);
                    const cx<T> om = mk((T)S.omega.x, (T)S.omega.y);
                    FOR_SITES
                    {
                        const int i = base + j_;
                        Spinor<T> pp, ss, tt, rh;
                        Spinor<TE> ee;
                        load_spinor<PE, false>(A.e, i, ee);
                        load_spinor<P, false>(A.p, i, pp);
                        load_spinor<P, false>(A.s, i, ss);
                        load_spinor<P, false>(A.t, i, tt);
#pragma unroll
                        for (int s = 0; s < 4; ++s)
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const cx<T> d = al * pp.c[s][c] + om * ss.c[s][c];
                                ee.c[s][c] = ee.c[s][c] + mk((TE)d.re, (TE)d.im);
                                ss.c[s][c] = ss.c[s][c] - om * tt.c[s][c];
                            }
                        store_spinor<PE>(A.e, i, ee);
                        store_spinor<P>(A.r, i, ss);
                        if (P == PREC16 || P == PRECBF) load_spinor<P, false>(A.r, i, ss);
                        load_spinor<P, false>(A.rh, i, rh);
                        cdot_acc(rh, ss, qr, qi);
                        qn += nrm_acc(ss);
                    }
                }
                reduce_put(A, qr, qi, qn, 3, rb);
                SYNC_OR_RETURN;
                gather_own(A, sys, 3, red, rb);
                if (tid == 0 && act2) {
                    S.it += 1;
                    S.itc += 1;
                    const double2 rn = make_double2(red[0], red[1]);
                    S.rr = red[2];
                    // the inner residual starts at 1: far above it, the
                    // low-precision recurrences have diverged; stop and keep
                    // the correction so far (the outer cycle recomputes the
                    // true residual)
                    if (S.idone == 2 || S.itc >= A.max_inner || S.it >= A.max_iter || !(S.rr > S.itol2) ||
                        !finite2(rn) || S.rr > 1e8) {
                        S.idone = 1;
                    } else {
                        S.beta = cmul(cdiv(rn, S.rho), cdiv(S.alpha, S.omega));
                        if (!finite2(S.beta)) S.idone = 1;
                        S.rho = rn;
                    }
                }
                if (tid == 0 && S.idone) S.idone = 1;
                __syncthreads();
            }
            // p = r + beta (p - omega v)
            if (act2 && !S.idone && WORDS) {
                const float2 be = make_float2((float)S.beta.x, (float)S.beta.y);
                const float2 mom = make_float2(-(float)S.omega.x, -(float)S.omega.y);
                FOR_WORDS
                {
                    WORD_ADDR;
                    W4(A.p)[a] = caxpy2(be, caxpy2(mom, W4(A.v)[a], W4(A.p)[a]), W4(A.r)[a]);
                }
            } else if (act2 && !S.idone) {
                const cx<T> be = mk((T)S.beta.x, (T)S.beta.y);
                const cx<T> om = mk((T)S.omega.x, (T)S.omega.y);
                FOR_SITES
                {
                    const int i = base + j_;
                    Spinor<T> r, pp, v;
                    load_spinor<P, false>(A.r, i, r);
                    load_spinor<P, false>(A.p, i, pp);
                    load_spinor<P, false>(A.v, i, v);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) r.c[s][c] = r.c[s][c] + be * (pp.c[s][c] - om * v.c[s][c]);
                    store_spinor<P>(A.p, i, r);
                }
            }
            SYNC_OR_RETURN;
        }
        }  // BiCGstab
        }  // inner solve (not SAP)

        // ---- x += |r64| e (double)
        if (S.active && WORDS) {
            const double sc = sqrt(S.rn2);
            double2* xx = (double2*)A.x.v;
            FOR_WORDS
            {
                const int k = f_ / A.nsite, i = base + (f_ % A.nsite);
                const float4 w = W4(A.e)[(size_t)k * A.g.Vh + i];
                double2* x0 = xx + (size_t)(2 * k) * A.g.Vh + i;
                double2* x1 = xx + (size_t)(2 * k + 1) * A.g.Vh + i;
                const double2 a0 = *x0, a1 = *x1;
                *x0 = make_double2(a0.x + sc * w.x, a0.y + sc * w.y);
                *x1 = make_double2(a1.x + sc * w.z, a1.y + sc * w.w);
            }
        } else if (S.active) {
            const double sc = sqrt(S.rn2);
            FOR_SITES
            {
                const int i = base + j_;
                Spinor<double> xx;
                Spinor<TE> ee;
                load_spinor<PREC64, false>(A.x, i, xx);
                load_spinor<PE, false>(A.e, i, ee);
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        xx.c[s][c] = xx.c[s][c] + mk(sc * (double)ee.c[s][c].re, sc * (double)ee.c[s][c].im);
                store_spinor<PREC64>(A.x, i, xx);
            }
        }
        SYNC_OR_RETURN;
        // ---- t64 = H_oe x (double)
        if (S.active) FOR_SITES
            {
                const int i = base + j_;
                Spinor<TR> a;
                hop_site<PR, false, SOLVE_UNR>(A.g, A.mode, 0, 1, i, A.x, A.U64, a);
                store_spinor<PT>(A.t64, i, a);
            }
        SYNC_OR_RETURN;
        // ---- r64 = b - x + k2 H_eo t64 ; |r64|^2
        {
            double q = 0.0;
            if (S.active) {
                FOR_SITES
                {
                    const int i = base + j_;
                    Spinor<double> a, xx, bb;
                    {
                        Spinor<TR> ha;
                        hop_site<PT, false, SOLVE_UNR>(A.g, A.mode, 0, 0, i, A.t64, A.U64, ha);
                        to_double(ha, a);
                    }
                    load_spinor<PREC64, false>(A.x, i, xx);
                    load_spinor<PREC64, true>(A.b, i, bb);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) a.c[s][c] = bb.c[s][c] - A.diag * xx.c[s][c] + A.k2 * a.c[s][c];
                    store_spinor<PREC64>(A.r64, i, a);
                    q += nrm_acc(a);
                }
            }
            reduce_put(A, q, 0.0, 0.0, 1, rb);
            SYNC_OR_RETURN;
            gather_own(A, sys, 1, red, rb);
            if (tid == 0 && S.active) S.rn2 = red[0];
            __syncthreads();
        }
    }

    if (leader) {
        A.iters[sys] = S.it;
        A.resid[sys] = S.bn2 > 0.0 ? sqrt(S.rn2 / S.bn2) : 0.0;
        if (sys == 0) *A.outer_out = outer;
        if (final_flag == F_NAN) atomicCAS(A.status, 0, LQCD_ERR_NAN);
        if (final_flag == F_MAXIT) atomicCAS(A.status, 0, LQCD_ERR_NOCONVERGE);
        if (final_flag == F_NAN) atomicCAS(A.sticky, 0, LQCD_ERR_NAN);
        if (final_flag == F_MAXIT) atomicCAS(A.sticky, 0, LQCD_ERR_NOCONVERGE);
        atomicAdd(A.acc, (unsigned long long)S.it);
        atomicAdd(A.acc + (A.method == SOLVER_SERIES ? 3 : (A.method == SOLVER_SAP || A.method == SOLVER_SAPB) ? 4 : 1),
                  (unsigned long long)S.it * (unsigned long long)A.nsite);
        atomicAdd(A.acc + 2, (unsigned long long)outer * (unsigned long long)A.nsite);
    }
}

#undef FOR_SITES
#undef FOR_WORDS
#undef WORD_ADDR
#undef W4
#undef SYNC_OR_RETURN

// ---------------------------------------------------------------------------
// The geometric series of the slab systems on thread-block clusters
//
// One cluster of CL_CTAS CTAs per system (one x0-slab or sub-slab), one CTA
// per SM.  The single-precision inner vectors of the series (the iterate p,
// the odd intermediate H_oe p and the inner source r) live in the CTAs'
// shared memory, each CTA holding a contiguous chunk of the system's sites;
// the hopping term reads a neighbour's spinor from the shared memory of the
// CTA that owns it (distributed shared memory), and the CTAs of a system
// meet at an mbarrier handshake inside the cluster instead of the global
// counter of k_solve.  The outer double defect correction (double-float
// residual sweeps on the double fields) is that of k_solve.  Every wait is
// bounded: a CTA that gives up records LQCD_ERR_TIMEOUT and skips to the
// end, where the cluster's CTAs meet once more before they exit (no CTA
// leaves while another may still read its shared memory).
// ---------------------------------------------------------------------------
constexpr int CL_CTAS = 16;     // CTAs per cluster (one system)
constexpr int CL_BS = 512;      // threads per CTA
constexpr int CL_CHUNK = 512;   // at most this many sites per CTA
constexpr int CL_VEC = 6 * CL_CHUNK;  // float4 words of one vector chunk

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// bounded barrier of the cluster: every CTA arrives (release, cluster
// scope) on every CTA's mbarrier, then waits on its own for the phase to
// complete; false when the wait gave up
__device__ bool cl_sync(const SolveArgs& A, unsigned long long* mbar, uint32_t& parity, int ncta)
{
    __shared__ int s_ok;
    __syncthreads();
    // thread r arrives on CTA r's barrier: the ncta releases run in parallel
    // (each orders the CTA's writes before it through the __syncthreads)
    const uint32_t local = smem_u32(mbar);
    if ((int)threadIdx.x < ncta) {
        uint32_t remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"((int)threadIdx.x));
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
    }
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        int ok = 0;
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(local), "r"(parity)
                : "memory");
            if (done) {
                ok = 1;
                break;
            }
            if (*(volatile int*)A.status == LQCD_ERR_TIMEOUT || clock64() - t0 > A.spin_limit) break;
        }
        if (!ok) {
            atomicExch(A.status, LQCD_ERR_TIMEOUT);
            atomicCAS(A.sticky, 0, LQCD_ERR_TIMEOUT);
        }
        parity ^= 1u;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// sum over the cluster of up to three doubles: the CTA's partial goes to
// its own slot, and after the barrier every CTA adds all slots in rank
// order (the same totals in every CTA).  Double-buffered like reduce_put.
__device__ bool cl_reduce(const SolveArgs& A, unsigned long long* mbar, uint32_t& parity, int ncta,
                          double (*slot)[NQ], int& rb, double a, double b, double c, int nq, double* out)
{
    namespace cg = cooperative_groups;
    __shared__ double sh[NQ][CL_BS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
        sh[2][w] = c;
    }
    __syncthreads();
    if ((int)threadIdx.x < nq) {
        double v = 0.0;
        for (int k = 0; k < CL_BS / 32; ++k) v += sh[threadIdx.x][k];
        slot[rb][threadIdx.x] = v;
    }
    if (!cl_sync(A, mbar, parity, ncta)) return false;
    if ((int)threadIdx.x < nq) {
        cg::cluster_group cl = cg::this_cluster();
        double v = 0.0;
        for (int r = 0; r < ncta; ++r) v += cl.map_shared_rank(&slot[rb][0], r)[threadIdx.x];
        out[threadIdx.x] = v;
    }
    rb ^= 1;
    __syncthreads();
    return true;
}

__global__ void __launch_bounds__(CL_BS, 1) k_series_cl(SolveArgs A)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int ncta = CL_CTAS;
    const int sys = blockIdx.x / CL_CTAS;
    const int tid = threadIdx.x;
    const bool leader = (rank == 0 && tid == 0);
    const int base = (A.slab0 + sys * A.slabstep) * A.g.Sh;
    const int chunk = A.chunk;
    const int j0 = rank * chunk, j1 = min(A.nsite, j0 + chunk);
    extern __shared__ __align__(16) float4 cl_dyn[];
    float4* ps = cl_dyn;              // iterate p, [6][CL_CHUNK]
    float4* ts = cl_dyn + CL_VEC;      // H_oe p
    float4* rs = cl_dyn + 2 * CL_VEC;  // inner source r
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ double slot[2][NQ];
    __shared__ SysSt S;
    __shared__ double red[NQ];
    __shared__ int s_fail;
    uint32_t parity = 0;
    int rb = 0;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(ncta) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    // every CTA's mbarrier exists before anyone arrives on it
    cl.sync();

    // spinor of eo index j (of the system's parity block) from the shared
    // memory of the CTA that owns it
    // (chunk a power of two: the owner by a shift; the own chunk read
    // directly, only the other CTAs' through the cluster window)
    const int lgc = (chunk & (chunk - 1)) == 0 ? __ffs(chunk) - 1 : -1;
    auto dsm = [&](const float4* buf, int j, Spinor<float>& sp) {
        const int loc = j - base;
        const int r = lgc >= 0 ? loc >> lgc : loc / chunk, off = loc - r * chunk;
        const float4* q = (r == rank ? buf : cl.map_shared_rank(buf, r)) + off;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 d = q[k * CL_CHUNK];
            sp.c[(2 * k) / 3][(2 * k) % 3] = mk(d.x, d.y);
            sp.c[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(d.z, d.w);
        }
    };
    auto st_loc = [&](float4* buf, int off, const Spinor<float>& sp) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const cx<float> a = sp.c[(2 * k) / 3][(2 * k) % 3], b = sp.c[(2 * k + 1) / 3][(2 * k + 1) % 3];
            buf[k * CL_CHUNK + off] = make_float4(a.re, a.im, b.re, b.im);
        }
    };
    auto ld_loc = [&](const float4* buf, int off, Spinor<float>& sp) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 d = buf[k * CL_CHUNK + off];
            sp.c[(2 * k) / 3][(2 * k) % 3] = mk(d.x, d.y);
            sp.c[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(d.z, d.w);
        }
    };
#define CL_SITES for (int j_ = j0 + tid; j_ < j1; j_ += CL_BS)
#define CL_SYNC_OR_END                                     \
    if (!cl_sync(A, &mbar, parity, ncta)) { \
        s_fail = 1;                                        \
        goto the_end;                                      \
    }
#define CL_REDUCE_OR_END(a, b, c, nq)                                                  \
    if (!cl_reduce(A, &mbar, parity, ncta, slot, rb, (a), (b), (c), (nq), red)) { \
        s_fail = 1;                                                                    \
        goto the_end;                                                                  \
    }
    {
        int outer = 0, final_flag = F_DONE;
        // ---- x = 0, r64 = b, |b|^2; with an initial guess: t64 = H_oe x
        {
            double q = 0.0;
            CL_SITES
            {
                const int i = base + j_;
                Spinor<double> bb, z;
                load_spinor<PREC64, true>(A.b, i, bb);
                if (A.guess) {
                    Spinor<df> hz;
                    hop_site<PRECDF, false, SOLVE_UNR>(A.g, A.mode, 0, 1, i, A.x, A.U64, hz);
                    store_spinor<PRECDS>(A.t64, i, hz);
                } else {
                    store_spinor<PREC64>(A.r64, i, bb);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) z.c[s][c] = mk(0.0, 0.0);
                    store_spinor<PREC64>(A.x, i, z);
                }
                q += nrm_acc(bb);
            }
            CL_REDUCE_OR_END(q, 0.0, 0.0, 1);
            if (tid == 0) {
                S.bn2 = red[0];
                S.rn2 = red[0];
                S.it = 0;
            }
            __syncthreads();
        }
        if (A.guess) {
            double q = 0.0;
            CL_SITES
            {
                const int i = base + j_;
                Spinor<double> a, xx, bb;
                {
                    Spinor<df> ha;
                    hop_site<PRECDS, false, SOLVE_UNR>(A.g, A.mode, 0, 0, i, A.t64, A.U64, ha);
                    to_double(ha, a);
                }
                load_spinor<PREC64, false>(A.x, i, xx);
                load_spinor<PREC64, true>(A.b, i, bb);
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) a.c[s][c] = bb.c[s][c] - A.diag * xx.c[s][c] + A.k2 * a.c[s][c];
                store_spinor<PREC64>(A.r64, i, a);
                q += nrm_acc(a);
            }
            CL_REDUCE_OR_END(q, 0.0, 0.0, 1);
            if (tid == 0) S.rn2 = red[0];
            __syncthreads();
            if (!(S.bn2 > 0.0)) CL_SITES
                {
                    Spinor<double> z;
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) z.c[s][c] = mk(0.0, 0.0);
                    store_spinor<PREC64>(A.x, base + j_, z);
                }
        }
        for (;;) {
            if (tid == 0) {
                const bool nan = !isfinite(S.rn2);
                const bool conv = !(S.rn2 > A.tol * A.tol * S.bn2) || !(S.bn2 > 0.0);
                S.active = (!nan && !conv) ? 1 : 0;
                int f = nan ? F_NAN : conv ? F_DONE : F_ACTIVE;
                if (f == F_ACTIVE && (outer >= A.max_outer || S.it >= A.max_iter)) f = F_MAXIT;
                S.flag = f;
            }
            __syncthreads();
            if (S.flag != F_ACTIVE) {
                final_flag = S.flag;
                break;
            }
            ++outer;
            // ---- inner start: r = p = r64 / |r64|
            {
                const double sc = 1.0 / sqrt(S.rn2);
                double q = 0.0;
                CL_SITES
                {
                    const int i = base + j_;
                    Spinor<double> r6;
                    load_spinor<PREC64, false>(A.r64, i, r6);
                    Spinor<float> r;
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            r.c[s][c] = mk((float)(sc * r6.c[s][c].re), (float)(sc * r6.c[s][c].im));
                    st_loc(rs, j_ - j0, r);
                    st_loc(ps, j_ - j0, r);
                    q += nrm_acc(r);
                }
                CL_REDUCE_OR_END(q, 0.0, 0.0, 1);
                if (tid == 0) {
                    S.idone = 0;
                    S.itc = 0;
                    const double need = 0.5 * A.tol * sqrt(S.bn2 / fmax(S.rn2, 1e-300));
                    const double it = fmax(A.inner_tol, need);
                    S.itol2 = it * it;
                }
                __syncthreads();
            }
            // ---- the series p <- (r + k2 H_eo H_oe p) / diag, its residual
            // reduced every second iteration (as in k_solve)
            {
                const float k2 = (float)A.k2, dinv = (float)(1.0 / A.diag);
                for (;;) {
                    if (S.idone) break;
                    const bool chk = (S.itc & 1) || S.itc + 1 >= A.max_inner || S.it + 1 >= A.max_iter;
                    CL_SITES
                    {
                        Spinor<float> a;
                        hop_site_ld<PREC32, SERIES_UNR>(A.g, A.mode, 0, 1, base + j_,
                                                        [&](int j, Spinor<float>& sp) { dsm(ps, j, sp); }, A.UP, a);
                        st_loc(ts, j_ - j0, a);
                    }
                    CL_SYNC_OR_END;
                    double q = 0.0;
                    CL_SITES
                    {
                        Spinor<float> a, pp, rr;
                        hop_site_ld<PREC32, SERIES_UNR>(A.g, A.mode, 0, 0, base + j_,
                                                        [&](int j, Spinor<float>& sp) { dsm(ts, j, sp); }, A.UP, a);
                        ld_loc(ps, j_ - j0, pp);
                        ld_loc(rs, j_ - j0, rr);
#pragma unroll
                        for (int s = 0; s < 4; ++s)
#pragma unroll
                            for (int c = 0; c < 3; ++c) a.c[s][c] = dinv * (rr.c[s][c] + k2 * a.c[s][c]);
                        st_loc(ps, j_ - j0, a);
                        if (chk) {
#pragma unroll
                            for (int s = 0; s < 4; ++s)
#pragma unroll
                                for (int c = 0; c < 3; ++c) pp.c[s][c] = a.c[s][c] - pp.c[s][c];
                            q += nrm_acc(pp);
                        }
                    }
                    if (!chk) {
                        CL_SYNC_OR_END;
                        if (tid == 0) {
                            S.it += 1;
                            S.itc += 1;
                        }
                        __syncthreads();
                        continue;
                    }
                    CL_REDUCE_OR_END(q, 0.0, 0.0, 1);
                    if (tid == 0) {
                        S.it += 1;
                        S.itc += 1;
                        const double res2 = A.diag * A.diag * red[0];
                        if (!(res2 > S.itol2) || S.itc >= A.max_inner || S.it >= A.max_iter) S.idone = 1;
                        if (!isfinite(res2) || (S.itc >= 16 && res2 > 1e6)) {
                            S.idone = 1;
                            S.it = A.max_iter;
                        }
                    }
                    __syncthreads();
                }
            }
            // ---- x += |r64| p (double)
            {
                const double sc = sqrt(S.rn2);
                CL_SITES
                {
                    const int i = base + j_;
                    Spinor<double> xx;
                    Spinor<float> e;
                    load_spinor<PREC64, false>(A.x, i, xx);
                    ld_loc(ps, j_ - j0, e);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            xx.c[s][c] = xx.c[s][c] + mk(sc * (double)e.c[s][c].re, sc * (double)e.c[s][c].im);
                    store_spinor<PREC64>(A.x, i, xx);
                }
            }
            CL_SYNC_OR_END;
            // ---- t64 = H_oe x (double-float)
            CL_SITES
            {
                const int i = base + j_;
                Spinor<df> a;
                hop_site<PRECDF, false, SOLVE_UNR>(A.g, A.mode, 0, 1, i, A.x, A.U64, a);
                store_spinor<PRECDS>(A.t64, i, a);
            }
            CL_SYNC_OR_END;
            // ---- r64 = b - diag x + k2 H_eo t64 ; |r64|^2
            {
                double q = 0.0;
                CL_SITES
                {
                    const int i = base + j_;
                    Spinor<double> a, xx, bb;
                    {
                        Spinor<df> ha;
                        hop_site<PRECDS, false, SOLVE_UNR>(A.g, A.mode, 0, 0, i, A.t64, A.U64, ha);
                        to_double(ha, a);
                    }
                    load_spinor<PREC64, false>(A.x, i, xx);
                    load_spinor<PREC64, true>(A.b, i, bb);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) a.c[s][c] = bb.c[s][c] - A.diag * xx.c[s][c] + A.k2 * a.c[s][c];
                    store_spinor<PREC64>(A.r64, i, a);
                    q += nrm_acc(a);
                }
                CL_REDUCE_OR_END(q, 0.0, 0.0, 1);
                if (tid == 0) S.rn2 = red[0];
                __syncthreads();
            }
        }
        if (leader) {
            A.iters[sys] = S.it;
            A.resid[sys] = S.bn2 > 0.0 ? sqrt(S.rn2 / S.bn2) : 0.0;
            if (sys == 0) *A.outer_out = outer;
            if (final_flag == F_NAN) atomicCAS(A.status, 0, LQCD_ERR_NAN);
            if (final_flag == F_MAXIT) atomicCAS(A.status, 0, LQCD_ERR_NOCONVERGE);
            if (final_flag == F_NAN) atomicCAS(A.sticky, 0, LQCD_ERR_NAN);
            if (final_flag == F_MAXIT) atomicCAS(A.sticky, 0, LQCD_ERR_NOCONVERGE);
            atomicAdd(A.acc, (unsigned long long)S.it);
            atomicAdd(A.acc + 3, (unsigned long long)S.it * (unsigned long long)A.nsite);
            atomicAdd(A.acc + 2, (unsigned long long)outer * (unsigned long long)A.nsite);
        }
    }
the_end:
    // no CTA leaves while another of its cluster may still read its shared
    // memory: every path (converged, failed, or a wait that gave up) ends here
    cl.sync();
}
#undef CL_SITES
#undef CL_SYNC_OR_END
#undef CL_REDUCE_OR_END

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Work {
    double2* vec[8] = {nullptr};  // inner vectors, each sized for a double half field
    double2* r64 = nullptr;
    double2* t64 = nullptr;
    double* part = nullptr;       // [2][NQ][grid] double-buffered partial sums
    unsigned* bar = nullptr;      // [NSYS_MAX][BAR_STRIDE] barrier counters
    int* status = nullptr;
    int* sticky = nullptr;  // int[4] then unsigned long long[NACC] (sticky status, iteration sums)
    int* iters = nullptr;
    double* resid = nullptr;
    int* outer = nullptr;
    int* h_status = nullptr;  // pinned mirror: status, outer, iters[NSYS_MAX]
    double* h_resid = nullptr;
    int gmax[NPREC] = {0, 0, 0, 0};  // co-resident CTAs per precision
    int cl_ok = 0;                   // the device runs k_series_cl's clusters
    // the Schwarz-preconditioned global solve: 11 full-lattice vectors, each
    // sized for a double full field (allocated on first use)
    static constexpr int NSAP = 11;
    double2* sap[NSAP] = {nullptr};
};

// parity block `par` of a full-lattice vector in precision prec (parity 0
// block, parity 1 block; for half storage the two scale arrays follow)
static SpinorF full_view(double2* buf, int prec, int par, int Vh)
{
    SpinorF f;
    f.N = Vh;
    f.nrm = nullptr;
    if (prec == PREC64) {
        f.v = buf + (size_t)par * 12 * Vh;
    } else if (prec == PREC32) {
        f.v = (float4*)buf + (size_t)par * 6 * Vh;
    } else {
        f.v = (uint4*)buf + (size_t)par * 3 * Vh;
        if (prec == PREC16) f.nrm = (float*)((uint4*)buf + (size_t)6 * Vh) + (size_t)par * Vh;
    }
    return f;
}

static SpinorF inner_view(double2* buf, int prec, int Vh)
{
    SpinorF f;
    f.v = buf;
    f.N = Vh;
    // half: the per-site scales follow the 3*Vh uint4 words
    f.nrm = prec == PREC16 ? (float*)((uint4*)buf + (size_t)3 * Vh) : nullptr;
    return f;
}

int solver_init(lqcd_ctx* h)
{
    Work* w = new Work();
    h->work = w;
    const int Vh = h->g.Vh;
    for (int k = 0; k < 8; ++k) LQ_CUDA(h, cudaMalloc(&w->vec[k], sizeof(double2) * 12 * (size_t)Vh));
    LQ_CUDA(h, cudaMalloc(&w->r64, sizeof(double2) * 12 * (size_t)Vh));
    LQ_CUDA(h, cudaMalloc(&w->t64, sizeof(double2) * 12 * (size_t)Vh));
    // co-resident CTAs of a cooperative launch: the smaller occupancy of the
    // two variants of each precision
    int occ[NPREC], occs[NPREC];
    LQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_solve<PREC64, false>, SBS, 0));
    LQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_solve<PREC32, false>, SBS, 0));
    LQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], k_solve<PREC16, false>, SBS, 0));
    LQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[3], k_solve<PRECBF, false>, SBS, 0));
    // the Schwarz variants run with the 4-D block preconditioner's dynamic
    // shared memory (opted in here, counted in their occupancy)
    const int smd = sapb_smem_bytes<double>(), smf = sapb_smem_bytes<float>();
    LQ_CUDA(h, cudaFuncSetAttribute(k_solve<PREC64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smd));
    LQ_CUDA(h, cudaFuncSetAttribute(k_solve<PREC32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf));
    LQ_CUDA(h, cudaFuncSetAttribute(k_solve<PREC16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf));
    LQ_CUDA(h, cudaFuncSetAttribute(k_solve<PRECBF, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf));
    LQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occs[0], k_solve<PREC64, true>, SBS, smd));
    LQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occs[1], k_solve<PREC32, true>, SBS, smf));
    LQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occs[2], k_solve<PREC16, true>, SBS, smf));
    LQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occs[3], k_solve<PRECBF, true>, SBS, smf));
    // the cluster series solver: 16-CTA clusters (a non-portable size) with
    // three vector chunks of shared memory each; unsupported -> not used
    {
        const int clsm = 3 * CL_VEC * (int)sizeof(float4);
        cudaLaunchConfig_t cc = {};
        cc.gridDim = dim3(CL_CTAS);
        cc.blockDim = dim3(CL_BS);
        cc.dynamicSmemBytes = clsm;
        cudaLaunchAttribute ca[1];
        ca[0].id = cudaLaunchAttributeClusterDimension;
        ca[0].val.clusterDim.x = CL_CTAS;
        ca[0].val.clusterDim.y = 1;
        ca[0].val.clusterDim.z = 1;
        cc.attrs = ca;
        cc.numAttrs = 1;
        int ncl = 0;
        if (cudaFuncSetAttribute(k_series_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, clsm) != cudaSuccess ||
            cudaFuncSetAttribute(k_series_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
            cudaOccupancyMaxActiveClusters(&ncl, (const void*)k_series_cl, &cc) != cudaSuccess)
            ncl = 0;
        cudaGetLastError();  // an unsupported configuration leaves no error behind
        w->cl_ok = ncl >= 1 ? 1 : 0;
    }
    int gm = 0;
    for (int k = 0; k < NPREC; ++k) {
        w->gmax[k] = std::max(1, std::min(occ[k], occs[k])) * h->num_sms;
        gm = std::max(gm, w->gmax[k]);
    }
    LQ_CUDA(h, cudaMalloc(&w->part, sizeof(double) * 2 * NQ * (size_t)gm));
    LQ_CUDA(h, cudaMalloc(&w->bar, sizeof(unsigned) * BAR_STRIDE * NSYS_MAX));
    LQ_CUDA(h, cudaMalloc(&w->status, sizeof(int) * 4));
    LQ_CUDA(h, cudaMalloc(&w->sticky, sizeof(int) * 4 + sizeof(unsigned long long) * NACC));
    LQ_CUDA(h, cudaMemset(w->sticky, 0, sizeof(int) * 4 + sizeof(unsigned long long) * NACC));
    LQ_CUDA(h, cudaMalloc(&w->iters, sizeof(int) * NSYS_MAX));
    LQ_CUDA(h, cudaMalloc(&w->resid, sizeof(double) * NSYS_MAX));
    LQ_CUDA(h, cudaMalloc(&w->outer, sizeof(int) * 4));
    LQ_CUDA(h, cudaMallocHost(&w->h_status, sizeof(int) * (NSYS_MAX + 4)));
    LQ_CUDA(h, cudaMallocHost(&w->h_resid, sizeof(double) * NSYS_MAX));
    return LQCD_OK;
}

// reads and clears the sticky status and the iteration sums of the solves
// run since the last call (synchronises the stream)
int solver_collect(lqcd_ctx* h, int64_t* iters, int64_t* site_iters, int64_t* outer_sites,
                   int64_t* series_sites, int64_t* sap_sites)
{
    Work* w = h->work;
    int hs[4];
    unsigned long long acc[NACC];
    LQ_CUDA(h, cudaMemcpyAsync(hs, w->sticky, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
    LQ_CUDA(h, cudaMemcpyAsync(acc, w->sticky + 4, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    LQ_CUDA(h, cudaMemsetAsync(w->sticky, 0, sizeof(int) * 4 + sizeof(acc), h->stream));
    if (iters) *iters = (int64_t)acc[0];
    if (site_iters) *site_iters = (int64_t)acc[1];
    if (outer_sites) *outer_sites = (int64_t)acc[2];
    if (series_sites) *series_sites = (int64_t)acc[3];
    if (sap_sites) *sap_sites = (int64_t)acc[4];
    if (hs[0] != 0) {
        h->err = hs[0] == LQCD_ERR_TIMEOUT ? "solver: grid barrier wait timed out"
                 : hs[0] == LQCD_ERR_NAN   ? "solver: non-finite residual"
                                           : "solver: no convergence";
        return hs[0];
    }
    return LQCD_OK;
}

void solver_free(lqcd_ctx* h)
{
    Work* w = h->work;
    if (!w) return;
    for (int k = 0; k < 8; ++k) cudaFree(w->vec[k]);
    cudaFree(w->r64);
    cudaFree(w->t64);
    for (int k = 0; k < Work::NSAP; ++k) cudaFree(w->sap[k]);
    cudaFree(w->part);
    cudaFree(w->bar);
    cudaFree(w->status);
    cudaFree(w->sticky);
    cudaFree(w->iters);
    cudaFree(w->resid);
    cudaFree(w->outer);
    cudaFreeHost(w->h_status);
    cudaFreeHost(w->h_resid);
    delete w;
    h->work = nullptr;
}

// algorithmic DRAM bytes per system site: one inner iteration and one outer
// cycle (each vector and the eight links moved once per phase)
void solver_site_bytes(int prec, int method, double* inner, double* outer, int nsap)
{
    const double sp = prec == PREC64 ? 192.0 : prec == PREC32 ? 96.0 : prec == PREC16 ? 52.0 : 48.0;
    const double lk = prec == PREC64 ? 1152.0 : prec == PREC32 ? 384.0 : 192.0;
    const double se = prec == PREC64 ? 192.0 : 96.0;
    // BiCGstab: 24 spinor passes, 4 half sweeps of links, solution r/w;
    // series: p, tmp, tmp, r, p, p (6 passes), 2 half sweeps of links;
    // Schwarz-preconditioned BiCGstab (per even site of the lattice, nsap
    // series terms): two preconditioner applications of (17 + 5 nsap)
    // spinor passes and (4 + 2 nsap) half sweeps of links each (slab solves
    // of both colours, the face update, the Wilson matrix), plus 28 passes
    // of vector updates and the solution r/w of both parities
    // 4-D block preconditioner: per application the source and the links
    // are read and the block solution written once (the series runs in
    // shared memory); the Wilson matrix and vector updates as above
    if (method == SOLVER_SAP)
        *inner = 2.0 * (17.0 + 5.0 * nsap) * sp + 28.0 * sp + 2.0 * (4.0 + 2.0 * nsap) * lk + 4.0 * se;
    else if (method == SOLVER_SAPB)
        *inner = 2.0 * (4.0 * sp + lk) + 4.0 * lk + 28.0 * sp + 4.0 * se;
    else
        *inner = method == SOLVER_SERIES ? 6.0 * sp + 2.0 * lk : 24.0 * sp + 4.0 * lk + 2.0 * se;
    *outer = (192.0 + 3.0 * sp + se) + (2.0 * 192.0 + se) + (2.0 * 192.0 + 1152.0) + (4.0 * 192.0 + 1152.0);
}

int solver_sap_alloc(lqcd_ctx* h)
{
    Work* w = h->work;
    for (int k = 0; k < Work::NSAP; ++k)
        if (!w->sap[k]) {
            if (h->capturing) {
                h->err = "the Schwarz-preconditioned solve's workspace must exist before a graph is recorded";
                return LQCD_ERR_STATE;
            }
            LQ_CUDA(h, cudaMalloc(&w->sap[k], sizeof(double2) * 24 * (size_t)h->g.Vh));
        }
    return LQCD_OK;
}

// block extents of the 4-D Schwarz preconditioner: 4 where L[mu] is a
// multiple of 4, else 2 (every extent is even)
static int sapb_geometry(lqcd_ctx* h, SolveArgs& A)
{
    const Geo& g = h->g;
    int bvol = 1;
    A.nblk = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (g.L[mu] % 2) {
            h->err = "the block Schwarz preconditioner needs even extents";
            return LQCD_ERR_GEOM;
        }
        A.bk[mu] = g.L[mu] % 4 == 0 ? 4 : 2;
        A.lbk[mu] = A.bk[mu] == 4 ? 2 : 1;
        A.nbk[mu] = g.L[mu] / A.bk[mu];
        A.nblk *= A.nbk[mu];
        bvol *= A.bk[mu];
    }
    A.bvh = bvol / 2;
    if (A.bvh > SAPB_BVH) {
        h->err = "Schwarz block larger than one CTA";
        return LQCD_ERR_GEOM;
    }
    return LQCD_OK;
}

int eo_solve(lqcd_ctx* h, int mode, int colour, int prec, double kappa, double2* x_e, const double2* b_e,
             double tol, int max_iter, int* iters_sys, double* resid_sys, double diag, int method, int guess)
{
    Work* w = h->work;
    const Geo& g = h->g;
    SolveArgs A;
    A.g = g;
    A.mode = mode;
    A.k2 = kappa * kappa;
    A.diag = diag;
    A.method = method;
    A.guess = guess;
    A.kappa = kappa;
    const bool sap = method == SOLVER_SAP || method == SOLVER_SAPB;
    if (sap && (mode != MODE_ALL || diag != 1.0)) {
        h->err = "the Schwarz-preconditioned solve is a whole-lattice solve of M";
        return LQCD_ERR_ARG;
    }
    A.nsap = h->sap_terms;
    int smem = 0;
    if (method == SOLVER_SAPB) {
        LQ_TRY(sapb_geometry(h, A));
        smem = prec == PREC64 ? sapb_smem_bytes<double>() : sapb_smem_bytes<float>();
    }
    if (mode == MODE_INTRA) {
        A.nsys = colour < 0 ? g.nb : g.nb / 2;
        A.slab0 = colour < 0 ? 0 : colour;
        A.slabstep = colour < 0 ? 1 : 2;
        A.nsite = g.Sh;
    } else {
        A.nsys = 1;
        A.slab0 = 0;
        A.slabstep = 1;
        A.nsite = g.Vh;
    }
    if (A.nsys > NSYS_MAX) {
        h->err = "too many slabs for one batched solve";
        return LQCD_ERR_GEOM;
    }
    const int want = (A.nsite + SBS - 1) / SBS;
    // CTAs per system: spt sites per thread, or (spt = 0) every co-resident
    // CTA, so that all SMs carry the same share (at least 32 sites per CTA)
    const int spt = h->tune.solve_spt[prec][mode == MODE_INTRA ? 0 : 1];
    A.cps = spt <= 0 ? std::max(1, std::min(w->gmax[prec] / A.nsys, (A.nsite + 31) / 32))
                     : std::max(1, std::min(w->gmax[prec] / A.nsys, (want + spt - 1) / spt));
    A.chunk = (A.nsite + A.cps - 1) / A.cps;
    const int G = A.cps * A.nsys;
    A.U64 = gauge_view(h, PREC64);
    A.UP = gauge_view(h, prec);
    A.b = sp64((double2*)b_e, 0, g.Vh);
    A.x = sp64(x_e, 0, g.Vh);
    A.r64 = sp64(w->r64, 0, g.Vh);
    A.t64 = sp64(w->t64, 0, g.Vh);
    A.r = inner_view(w->vec[0], prec, g.Vh);
    A.rh = inner_view(w->vec[1], prec, g.Vh);
    A.p = inner_view(w->vec[2], prec, g.Vh);
    A.v = inner_view(w->vec[3], prec, g.Vh);
    A.s = inner_view(w->vec[4], prec, g.Vh);
    A.t = inner_view(w->vec[5], prec, g.Vh);
    A.tmp = inner_view(w->vec[6], prec, g.Vh);
    A.e = inner_view(w->vec[7], prec == PREC64 ? PREC64 : PREC32, g.Vh);
    if (sap) {
        LQ_TRY(solver_sap_alloc(h));
        SpinorF* fv[Work::NSAP] = {A.fr, A.frh, A.fp, A.fv, A.fs, A.ft, A.fzp, A.fzs, A.fw1, A.fw2, A.fy};
        for (int k = 0; k < Work::NSAP; ++k)
            for (int par = 0; par < 2; ++par)
                fv[k][par] = full_view(w->sap[k], k == Work::NSAP - 1 ? (prec == PREC64 ? PREC64 : PREC32) : prec,
                                       par, g.Vh);
        A.e = A.fy[0];  // the inner solution's even block
    }
    A.tol = tol;
    // inner relative residual: a few unit roundoffs of the storage
    // (bfloat16 keeps 8 significant bits, 2^-9 = 2e-3)
    // (bfloat16 keeps 8 significant bits: its Krylov recurrences drift from
    // the true residual within tens of iterations, so its inner solves stop
    // early and leave more of the reduction to the double outer cycles)
    A.inner_tol = prec == PREC64 ? 0.0 : prec == PREC32 ? 1e-5 : prec == PREC16 ? 2e-3 : 3e-2;
    A.max_iter = max_iter;
    A.max_outer = prec == PREC64 ? 8 : prec == PRECBF ? 80 : 40;
    A.max_inner = prec == PREC64 ? max_iter : prec == PREC32 ? 4000 : prec == PREC16 ? 600 : 200;
    A.part = w->part;
    A.bar = w->bar;
    A.status = w->status;
    A.sticky = w->sticky;
    A.acc = (unsigned long long*)(w->sticky + 4);
    A.iters = w->iters;
    A.resid = w->resid;
    A.outer_out = w->outer;
    A.spin_limit = h->wait_limit;
    LQ_CUDA(h, cudaMemsetAsync(w->bar, 0, sizeof(unsigned) * BAR_STRIDE * A.nsys, h->stream));
    LQ_CUDA(h, cudaMemsetAsync(w->status, 0, sizeof(int) * 4, h->stream));
    void* args[] = {&A};
    // the geometric series of single-precision slab systems of at most
    // CL_CTAS * CL_CHUNK sites runs on thread-block clusters (k_series_cl)
    const bool clu = w->cl_ok && h->tune.cluster_series && prec == PREC32 && method == SOLVER_SERIES &&
                     mode == MODE_INTRA && A.nsite <= CL_CTAS * CL_CHUNK;
    cudaEvent_t ev = nullptr;
    if (clu) {
        A.cps = CL_CTAS;
        A.chunk = (A.nsite + CL_CTAS - 1) / CL_CTAS;
        prof_begin(h, 1, &ev);
        cudaLaunchConfig_t cc = {};
        cc.gridDim = dim3(A.nsys * CL_CTAS);
        cc.blockDim = dim3(CL_BS);
        cc.dynamicSmemBytes = 3 * CL_VEC * sizeof(float4);
        cc.stream = h->stream;
        cudaLaunchAttribute ca[1];
        ca[0].id = cudaLaunchAttributeClusterDimension;
        ca[0].val.clusterDim.x = CL_CTAS;
        ca[0].val.clusterDim.y = 1;
        ca[0].val.clusterDim.z = 1;
        cc.attrs = ca;
        cc.numAttrs = 1;
        LQ_CUDA(h, cudaLaunchKernelExC(&cc, (const void*)k_series_cl, args));
        prof_end(h, 1, ev, 0.0);
    }
    const void* fn = prec == PREC64 ? (sap ? (const void*)k_solve<PREC64, true> : (const void*)k_solve<PREC64, false>)
                     : prec == PREC32 ? (sap ? (const void*)k_solve<PREC32, true> : (const void*)k_solve<PREC32, false>)
                     : prec == PREC16 ? (sap ? (const void*)k_solve<PREC16, true> : (const void*)k_solve<PREC16, false>)
                                      : (sap ? (const void*)k_solve<PRECBF, true> : (const void*)k_solve<PRECBF, false>);
    if (!clu) prof_begin(h, 1, &ev);
    // cooperative launch (every CTA resident), expressed as a launch
    // attribute so that it can also be recorded into a CUDA graph
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(SBS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (!clu) {
        LQ_CUDA(h, cudaLaunchKernelExC(&cfg, fn, args));
        prof_end(h, 1, ev, 0.0);
    }
    h->launches += 1;
    h->solve_count += 1;
    // deferred mode (graph capture): status and iterations stay on the
    // device (sticky status, iteration sums) until solver_collect
    if (h->deferred) return LQCD_OK;
    const size_t rec = h->prof.recs.size();
    LQ_CUDA(h, cudaMemcpyAsync(w->h_status, w->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LQ_CUDA(h, cudaMemcpyAsync(w->h_status + 1, w->outer, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LQ_CUDA(h, cudaMemcpyAsync(w->h_status + 4, w->iters, sizeof(int) * A.nsys, cudaMemcpyDeviceToHost,
                               h->stream));
    LQ_CUDA(h, cudaMemcpyAsync(w->h_resid, w->resid, sizeof(double) * A.nsys, cudaMemcpyDeviceToHost,
                               h->stream));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    const int st = w->h_status[0];
    const int nouter = w->h_status[1];
    double bi, bo;
    solver_site_bytes(prec, method, &bi, &bo, A.nsap);
    int64_t itsum = 0;
    for (int s = 0; s < A.nsys; ++s) {
        itsum += w->h_status[4 + s];
        if (iters_sys) iters_sys[s] = w->h_status[4 + s];
        if (resid_sys) resid_sys[s] = w->h_resid[s];
    }
    if (ev && rec > 0 && rec <= h->prof.recs.size())
        h->prof.recs[rec - 1].bytes = (double)A.nsite * ((double)itsum * bi + (double)nouter * A.nsys * bo);
    h->iter_count += itsum;
    h->site_iters += itsum * (int64_t)A.nsite;
    h->hop_sites += itsum * (int64_t)A.nsite * solver_hops_per_iter(method, A.nsap);
    if (st == LQCD_ERR_TIMEOUT) {
        h->err = "solver: grid barrier wait timed out";
        return LQCD_ERR_TIMEOUT;
    }
    if (st == LQCD_ERR_NAN) {
        h->err = "solver: non-finite residual";
        return LQCD_ERR_NAN;
    }
    if (st == LQCD_ERR_NOCONVERGE) {
        int mx = 0;
        double rmax = 0.0;
        for (int s = 0; s < A.nsys; ++s) {
            mx = std::max(mx, w->h_status[4 + s]);
            rmax = std::max(rmax, w->h_resid[s]);
        }
        char buf[160];
        snprintf(buf, sizeof(buf), "solver: no convergence (prec %d, %d outer cycles, %d inner iterations, residual %.3e)",
                 prec, nouter, mx, rmax);
        h->err = buf;
        return LQCD_ERR_NOCONVERGE;
    }
    return LQCD_OK;
}
