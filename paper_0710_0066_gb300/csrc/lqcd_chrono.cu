// lqcd_chrono.cu -- minimal-residual chronological guesses for the
// whole-lattice solves of the molecular dynamics (lqcd_hmc_params.chrono =
// 3): the initial guess of a solve A x = b is the combination
// x_0 = sum_i c_i v_i of the n most recent solutions v_i of the same solve
// site that minimises |b - A x_0| (the chronological inverter by minimal
// residual extrapolation of Brower, Ivanenko, Levi and Orginos, Nucl. Phys.
// B 484 (1997) 353).  A = 1 - kappa^2 H_eo H_oe is applied to the v_i with
// the single-precision links, the normal equations
//   sum_j <A v_i, A v_j> c_j = <A v_i, b>
// are reduced in double and solved on the device (Cholesky that drops the
// directions whose pivot falls below 1e-10 of the largest diagonal entry:
// nearly dependent previous solutions), and the guess is combined from the
// double-precision solutions.  The guess only has to be good: the solve's
// double defect correction starts from its exact residual.  Every step is a
// kernel that reads its scalars from device memory, so the whole guess can
// be recorded into the MD's CUDA graph.
#include <math.h>

#include "lqcd_common.cuh"

namespace {

constexpr int BS = 256;
constexpr int DOT_BLOCKS = 64;
constexpr int NACC = 2 * (lqcd_ctx::NMRE + 1);  // G_ij (j = 0..NMRE-1) and r_i, re and im

struct MreVecs {
    const float4* w[lqcd_ctx::NMRE];  // A v_i, single-precision even halves [6][Vh]
};
struct MreSrc {
    const double2* s[lqcd_ctx::NMRE];  // the kept solutions, double even halves [12][Vh]
};

// v = gamma5^g5 s as a single-precision even half ([12][Vh] double2 ->
// [6][Vh] float4)
__global__ void k_mre_load(float4* v, const double2* s, int Vh, int g5)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= (int64_t)6 * Vh) return;
    const int k = (int)(f / Vh), i = (int)(f - (int64_t)k * Vh);
    const double sg = (g5 && k >= 3) ? -1.0 : 1.0;  // words 3..5 hold spins 2, 3
    const double2 a = s[(size_t)(2 * k) * Vh + i], b = s[(size_t)(2 * k + 1) * Vh + i];
    v[f] = make_float4((float)(sg * a.x), (float)(sg * a.y), (float)(sg * b.x), (float)(sg * b.y));
}

// partial sums, per block and row i = blockIdx.y, of <w_i, w_j> (j >= i)
// and <w_i, b>: single-precision products per word, double accumulation
__global__ void __launch_bounds__(BS) k_mre_dots(MreVecs W, const double2* b, int n, int Vh, double* part)
{
    const int i = blockIdx.y;
    double acc[NACC];
#pragma unroll
    for (int q = 0; q < NACC; ++q) acc[q] = 0.0;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < (int64_t)6 * Vh;
         f += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = W.w[i][f];
#pragma unroll
        for (int j = 0; j < lqcd_ctx::NMRE; ++j) {
            if (j < i || j >= n) continue;
            const float4 c = W.w[j][f];
            acc[2 * j] += (double)(a.x * c.x + a.y * c.y + a.z * c.z + a.w * c.w);
            acc[2 * j + 1] += (double)(a.x * c.y - a.y * c.x + a.z * c.w - a.w * c.z);
        }
        const int k = (int)(f / Vh), s = (int)(f - (int64_t)k * Vh);
        const double2 b0 = b[(size_t)(2 * k) * Vh + s], b1 = b[(size_t)(2 * k + 1) * Vh + s];
        acc[NACC - 2] += a.x * b0.x + a.y * b0.y + a.z * b1.x + a.w * b1.y;
        acc[NACC - 1] += a.x * b0.y - a.y * b0.x + a.z * b1.y - a.w * b1.x;
    }
    __shared__ double sh[BS / 32][NACC];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NACC; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) sh[w][q] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < NACC) {
        double v = 0.0;
        for (int k = 0; k < BS / 32; ++k) v += sh[k][threadIdx.x];
        part[((size_t)i * gridDim.x + blockIdx.x) * NACC + threadIdx.x] = v;
    }
}

// the partials summed in block order; G Hermitian, then the minimal-residual
// coefficients c by a Cholesky factorisation that drops directions whose
// pivot is below 1e-10 of the largest diagonal entry (and gives c = 0 if
// anything is not finite).  One thread: n <= NMRE.
__global__ void k_mre_solve(const double* part, int nblocks, int n, double2* cout)
{
    if (threadIdx.x != 0) return;
    constexpr int N = lqcd_ctx::NMRE;
    double2 G[N][N], r[N], L[N][N], y[N], c[N];
    bool keep[N];
    bool ok = true;
    for (int i = 0; i < n; ++i) {
        double acc[NACC];
        for (int q = 0; q < NACC; ++q) acc[q] = 0.0;
        for (int blk = 0; blk < nblocks; ++blk)
            for (int q = 0; q < NACC; ++q) acc[q] += part[((size_t)i * nblocks + blk) * NACC + q];
        for (int j = i; j < n; ++j) {
            G[i][j] = make_double2(acc[2 * j], acc[2 * j + 1]);
            G[j][i] = make_double2(acc[2 * j], -acc[2 * j + 1]);
        }
        G[i][i].y = 0.0;
        r[i] = make_double2(acc[NACC - 2], acc[NACC - 1]);
    }
    double gmax = 0.0;
    for (int i = 0; i < n; ++i) gmax = fmax(gmax, G[i][i].x);
    if (!(gmax > 0.0) || !isfinite(gmax)) ok = false;
    for (int i = 0; i < N; ++i) {
        keep[i] = false;
        for (int m = 0; m < N; ++m) L[i][m] = make_double2(0.0, 0.0);
    }
    for (int k = 0; k < n && ok; ++k) {
        double d = G[k][k].x;
        for (int m = 0; m < k; ++m) d -= L[k][m].x * L[k][m].x + L[k][m].y * L[k][m].y;
        if (!isfinite(d)) { ok = false; break; }
        keep[k] = d > 1e-10 * gmax;
        if (!keep[k]) {
            for (int i = k + 1; i < n; ++i) L[i][k] = make_double2(0.0, 0.0);
            continue;
        }
        const double lk = sqrt(d);
        L[k][k] = make_double2(lk, 0.0);
        for (int i = k + 1; i < n; ++i) {
            // L_ik = (G_ik - sum_m L_im conj(L_km)) / L_kk
            double2 s = G[i][k];
            for (int m = 0; m < k; ++m) {
                s.x -= L[i][m].x * L[k][m].x + L[i][m].y * L[k][m].y;
                s.y -= L[i][m].y * L[k][m].x - L[i][m].x * L[k][m].y;
            }
            L[i][k] = make_double2(s.x / lk, s.y / lk);
        }
    }
    // L y = r, then L^dag c = y, over the kept directions
    for (int k = 0; k < n && ok; ++k) {
        if (!keep[k]) { y[k] = make_double2(0.0, 0.0); continue; }
        double2 s = r[k];
        for (int m = 0; m < k; ++m) {
            s.x -= L[k][m].x * y[m].x - L[k][m].y * y[m].y;
            s.y -= L[k][m].x * y[m].y + L[k][m].y * y[m].x;
        }
        y[k] = make_double2(s.x / L[k][k].x, s.y / L[k][k].x);
    }
    for (int k = n - 1; k >= 0 && ok; --k) {
        if (!keep[k]) { c[k] = make_double2(0.0, 0.0); continue; }
        double2 s = y[k];
        for (int m = k + 1; m < n; ++m) {  // conj(L_mk) c_m
            s.x -= L[m][k].x * c[m].x + L[m][k].y * c[m].y;
            s.y -= L[m][k].x * c[m].y - L[m][k].y * c[m].x;
        }
        c[k] = make_double2(s.x / L[k][k].x, s.y / L[k][k].x);
        if (!isfinite(c[k].x) || !isfinite(c[k].y)) ok = false;
    }
    for (int k = 0; k < n; ++k) cout[k] = ok ? c[k] : make_double2(0.0, 0.0);
}

// x = gamma5^g5 sum_i c_i s_i on the even half ([12][Vh] double2)
__global__ void k_mre_combine(double2* x, MreSrc S, const double2* c, int n, int Vh, int g5)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)12 * Vh) return;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < lqcd_ctx::NMRE; ++i) {
        if (i >= n) break;
        const double2 a = c[i], v = S.s[i][t];
        acc.x += a.x * v.x - a.y * v.y;
        acc.y += a.x * v.y + a.y * v.x;
    }
    const double sg = (g5 && (int)(t / Vh) >= 6) ? -1.0 : 1.0;  // spins 2, 3
    x[t] = make_double2(sg * acc.x, sg * acc.y);
}

inline int nblk(int64_t n) { return (int)((n + BS - 1) / BS); }

int check_launch(lqcd_ctx* h)
{
    h->launches += 1;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->err = std::string("chronological guess kernel: ") + cudaGetErrorString(e);
        return LQCD_ERR_CUDA;
    }
    return LQCD_OK;
}

}  // namespace

int chrono_mre_alloc(lqcd_ctx* h)
{
    const size_t half32 = sizeof(float4) * 6 * (size_t)h->g.Vh;
    for (int i = 0; i < lqcd_ctx::NMRE; ++i)
        if (!h->mre_w[i]) LQ_CUDA(h, cudaMalloc(&h->mre_w[i], half32));
    if (!h->mre_v) LQ_CUDA(h, cudaMalloc(&h->mre_v, half32));
    if (!h->mre_o) LQ_CUDA(h, cudaMalloc(&h->mre_o, half32));
    if (!h->mre_c) LQ_CUDA(h, cudaMalloc(&h->mre_c, sizeof(double2) * lqcd_ctx::NMRE));
    if (!h->mre_part)
        LQ_CUDA(h, cudaMalloc(&h->mre_part, sizeof(double) * lqcd_ctx::NMRE * DOT_BLOCKS * NACC));
    return LQCD_OK;
}

void chrono_mre_free(lqcd_ctx* h)
{
    for (float4*& p : h->mre_w) {
        cudaFree(p);
        p = nullptr;
    }
    cudaFree(h->mre_v);
    cudaFree(h->mre_o);
    cudaFree(h->mre_c);
    cudaFree(h->mre_part);
    h->mre_v = h->mre_o = nullptr;
    h->mre_c = nullptr;
    h->mre_part = nullptr;
}

int chrono_mre_guess(lqcd_ctx* h, const double2* const* sol, int n, double2* x_e, const double2* b_e, double kappa,
                     int dag)
{
    const Geo& g = h->g;
    const int Vh = g.Vh;
    if (n <= 0 || n > lqcd_ctx::NMRE || !h->mre_c) {
        h->err = "chronological guess: no minimal-residual workspace";
        return LQCD_ERR_STATE;
    }
    SpinorF v, o;
    v.v = h->mre_v;
    v.nrm = nullptr;
    v.N = Vh;
    o = v;
    o.v = h->mre_o;
    MreVecs W;
    MreSrc S;
    for (int i = 0; i < lqcd_ctx::NMRE; ++i) {
        W.w[i] = h->mre_w[i];
        S.s[i] = i < n ? sol[i] : nullptr;
    }
    for (int i = 0; i < n; ++i) {
        // w_i = (1 - kappa^2 H_eo H_oe) gamma5^dag s_i in single precision
        k_mre_load<<<nblk((int64_t)6 * Vh), BS, 0, h->stream>>>(h->mre_v, sol[i], Vh, dag);
        LQ_TRY(check_launch(h));
        SpinorF w = v;
        w.v = h->mre_w[i];
        LQ_TRY(hop_sweep(h, PREC32, MODE_ALL, 0, 1, -1, o, v, 0.0, SpinorF{nullptr, nullptr, 0}, 1.0));
        LQ_TRY(hop_sweep(h, PREC32, MODE_ALL, 0, 0, -1, w, o, 1.0, v, -kappa * kappa));
    }
    k_mre_dots<<<dim3(DOT_BLOCKS, n), BS, 0, h->stream>>>(W, b_e, n, Vh, h->mre_part);
    LQ_TRY(check_launch(h));
    k_mre_solve<<<1, 32, 0, h->stream>>>(h->mre_part, DOT_BLOCKS, n, h->mre_c);
    LQ_TRY(check_launch(h));
    k_mre_combine<<<nblk((int64_t)12 * Vh), BS, 0, h->stream>>>(x_e, S, h->mre_c, n, Vh, dag);
    return check_launch(h);
}
