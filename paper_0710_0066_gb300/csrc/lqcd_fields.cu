// lqcd_fields.cu -- layout conversion, index maps, boundary (Schur) space,
// BLAS-1, deterministic reductions and the Philox heatbath generator.
#include <math.h>

#include "lqcd_common.cuh"

namespace {

constexpr int BS = 256;

inline int nblk(int64_t n, int bs = BS) { return (int)((n + bs - 1) / bs); }

// ---------------------------------------------------------------------------
// spinors: ABI [site][4][3] complex (checkerboard order) <-> [par][12][Vh]
// ---------------------------------------------------------------------------
__global__ void k_pack_spinor(double2* dst, const double2* abi, int Vh, int par0, int npar)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)npar * Vh) return;
    const int q = (int)(t / Vh), i = (int)(t % Vh);
    const double2* a = abi + ((int64_t)q * Vh + i) * 12;
    double2* d = dst + (size_t)(par0 + q) * 12 * Vh;
#pragma unroll
    for (int c = 0; c < 12; ++c) d[(size_t)c * Vh + i] = a[c];
}

__global__ void k_unpack_spinor(double2* abi, const double2* src, int Vh, int par0, int npar)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)npar * Vh) return;
    const int q = (int)(t / Vh), i = (int)(t % Vh);
    double2* a = abi + ((int64_t)q * Vh + i) * 12;
    const double2* s = src + (size_t)(par0 + q) * 12 * Vh;
#pragma unroll
    for (int c = 0; c < 12; ++c) a[c] = s[(size_t)c * Vh + i];
}

template <int PS, int PD>
__global__ void k_convert(SpinorF dst, SpinorF src, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Spinor<typename Real<PS>::T> a;
    load_spinor<PS>(src, i, a);
    Spinor<typename Real<PD>::T> b;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            b.c[s][c] = mk((typename Real<PD>::T)a.c[s][c].re, (typename Real<PD>::T)a.c[s][c].im);
    store_spinor<PD>(dst, i, b);
}

// ---------------------------------------------------------------------------
// gauge: ABI [mu][site][3][3] -> double / single / half internal copies
// ---------------------------------------------------------------------------
__global__ void k_pack_gauge(double2* U64, float4* U32, uint2* U16, const double2* abi, int Vh)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)8 * Vh) return;
    const int mp = (int)(t / Vh), i = (int)(t % Vh);  // mp = mu*2 + parity
    const int mu = mp / 2, par = mp % 2;
    const double2* a = abi + ((int64_t)mu * 2 * Vh + (int64_t)par * Vh + i) * 9;
    double2 m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = a[k];
    double2* d64 = U64 + (size_t)mp * 9 * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) d64[(size_t)k * Vh + i] = m[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double2 x = m[2 * k], y = m[2 * k + 1];
        store_low_link_word(U32, U16, Vh, mp, k, i, x.x, x.y, y.x, y.y);
    }
}

__global__ void k_refresh_low(const double2* U64, float4* U32, uint2* U16, int Vh)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)8 * Vh) return;
    const int mp = (int)(t / Vh), i = (int)(t % Vh);
    const double2* s64 = U64 + (size_t)mp * 9 * Vh;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double2 x = s64[(size_t)(2 * k) * Vh + i], y = s64[(size_t)(2 * k + 1) * Vh + i];
        store_low_link_word(U32, U16, Vh, mp, k, i, x.x, x.y, y.x, y.y);
    }
}

__global__ void k_unpack_gauge(double2* abi, const double2* U64, int Vh)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)8 * Vh) return;
    const int mp = (int)(t / Vh), i = (int)(t % Vh);
    const int mu = mp / 2, par = mp % 2;
    double2* a = abi + ((int64_t)mu * 2 * Vh + (int64_t)par * Vh + i) * 9;
    const double2* s = U64 + (size_t)mp * 9 * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = s[(size_t)k * Vh + i];
}

// ---------------------------------------------------------------------------
// index maps (device computation from the geometry alone)
// ---------------------------------------------------------------------------
__device__ int site_cb(const Geo& g, const int x[4])
{
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    return p * g.Vh + (lex_of(g, x) >> 1);
}

__global__ void k_index_maps(int32_t* m, Geo g)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const int p = s >= g.Vh ? 1 : 0, i = s - p * g.Vh;
    int x[4];
    eo_coords(g, p, i, x);
    const int slab = x[0] / g.l0;
    m[0 * (size_t)g.V + s] = lex_of(g, x);
    m[1 * (size_t)g.V + s] = p;
    m[2 * (size_t)g.V + s] = slab;
    m[3 * (size_t)g.V + s] = slab & 1;
    for (int mu = 0; mu < 4; ++mu) {
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[mu] = (x[mu] + 1 == g.L[mu]) ? 0 : x[mu] + 1;
        m[(4 + mu) * (size_t)g.V + s] = site_cb(g, y);
        y[mu] = (x[mu] == 0) ? g.L[mu] - 1 : x[mu] - 1;
        m[(8 + mu) * (size_t)g.V + s] = site_cb(g, y);
    }
    const int first = (x[0] % g.l0) == 0;
    const int last = (x[0] % g.l0) == g.l0 - 1;
    m[12 * (size_t)g.V + s] = first | (last << 1);
    int b = -1;
    if ((slab & 1) && (first || last)) {
        const int lex3 = (x[1] * g.L[2] + x[2]) * g.L[3] + x[3];
        b = ((slab >> 1) * 2 + (first ? 0 : 1)) * g.V3 + lex3;
    }
    m[13 * (size_t)g.V + s] = b;
}

// ---------------------------------------------------------------------------
// boundary space: coords [nb/2][2][V3][2][3] <-> full internal field
// face 0 basis (e_i - e_{i+2})/sqrt2, face 1 basis (e_i + e_{i+2})/sqrt2
// ---------------------------------------------------------------------------
__device__ void face_site(const Geo& g, int j, int f, int lex3, int& par, int& i)
{
    int x[4];
    x[0] = (2 * j + 1) * g.l0 + (f ? g.l0 - 1 : 0);
    x[3] = lex3 % g.L[3];
    x[2] = (lex3 / g.L[3]) % g.L[2];
    x[1] = lex3 / (g.L[3] * g.L[2]);
    par = (x[0] + x[1] + x[2] + x[3]) & 1;
    i = lex_of(g, x) >> 1;
}

// one thread per (j, lex3); both faces (they coincide for l0 = 1), or only
// face 0 when nface = 1 (second level: coords [nb/2][V3][2][3])
__global__ void k_embed(double2* full, const double2* coords, Geo g, int nface)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nj = g.nb / 2;
    if (t >= nj * g.V3) return;
    const int j = t / g.V3, l3 = t % g.V3;
    const double r = 0.70710678118654752440;
    double2 out[2][12];
    int par[2], idx[2];
    for (int f = 0; f < nface; ++f) {
        face_site(g, j, f, l3, par[f], idx[f]);
        const double2* c = coords + ((size_t)(j * nface + f) * g.V3 + l3) * 6;
        const double sgn = f ? 1.0 : -1.0;
        for (int s = 0; s < 2; ++s)
            for (int col = 0; col < 3; ++col) {
                const double2 v = c[s * 3 + col];
                out[f][s * 3 + col] = make_double2(r * v.x, r * v.y);
                out[f][(s + 2) * 3 + col] = make_double2(sgn * r * v.x, sgn * r * v.y);
            }
    }
    if (g.l0 == 1 && nface == 2) {
        double2* d = full + (size_t)par[0] * 12 * g.Vh;
        for (int c = 0; c < 12; ++c)
            d[(size_t)c * g.Vh + idx[0]] = make_double2(out[0][c].x + out[1][c].x, out[0][c].y + out[1][c].y);
    } else {
        for (int f = 0; f < nface; ++f) {
            double2* d = full + (size_t)par[f] * 12 * g.Vh;
            for (int c = 0; c < 12; ++c) d[(size_t)c * g.Vh + idx[f]] = out[f][c];
        }
    }
}

__global__ void k_project(double2* coords, const double2* full, Geo g, int nface)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nj = g.nb / 2;
    if (t >= nj * nface * g.V3) return;
    const int jf = t / g.V3, l3 = t % g.V3;
    const int j = jf / nface, f = jf % nface;
    int par, i;
    face_site(g, j, f, l3, par, i);
    const double2* s = full + (size_t)par * 12 * g.Vh;
    const double r = 0.70710678118654752440;
    const double sgn = f ? 1.0 : -1.0;
    double2* c = coords + ((size_t)jf * g.V3 + l3) * 6;
    for (int sp = 0; sp < 2; ++sp)
        for (int col = 0; col < 3; ++col) {
            const double2 u = s[(size_t)(sp * 3 + col) * g.Vh + i];
            const double2 d = s[(size_t)((sp + 2) * 3 + col) * g.Vh + i];
            c[sp * 3 + col] = make_double2(r * (u.x + sgn * d.x), r * (u.y + sgn * d.y));
        }
}

// ---------------------------------------------------------------------------
// BLAS-1 on full double fields [2][12][Vh] (colour mask on the slab)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int slab_of_eo(const Geo& g, int i) { return ((2 * i) / g.V3) / g.l0; }

__global__ void k_axpby(double2* y, double a, const double2* x, double b, Geo g, int colour)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)24 * g.Vh) return;
    const int i = (int)(t % g.Vh);
    if (colour >= 0 && (slab_of_eo(g, i) & 1) != colour) {
        y[t] = make_double2(0.0, 0.0);
        return;
    }
    const double2 xv = x ? x[t] : make_double2(0.0, 0.0);
    const double2 yv = (b != 0.0) ? y[t] : make_double2(0.0, 0.0);
    y[t] = make_double2(a * xv.x + b * yv.x, a * xv.y + b * yv.y);
}

__global__ void k_gamma5(double2* y, const double2* x, int Vh)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)24 * Vh) return;
    const int comp = (int)((t / Vh) % 12);
    const double s = comp >= 6 ? -1.0 : 1.0;  // spins 2, 3
    const double2 v = x[t];
    y[t] = make_double2(s * v.x, s * v.y);
}

__global__ void k_lincomb_even(double2* y, double a, const double2* x1, double b, const double2* x0, int Vh, int g5)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)12 * Vh) return;
    const double s = (g5 && (int)(t / Vh) >= 6) ? -1.0 : 1.0;  // spins 2, 3
    const double2 u = x1[t];
    const double2 v = (b != 0.0) ? x0[t] : make_double2(0.0, 0.0);
    y[t] = make_double2(s * (a * u.x + b * v.x), s * (a * u.y + b * v.y));
}

__global__ void k_lincomb3_even(double2* y, double a, const double2* x2, double b, const double2* x1, double c,
                                const double2* x0, int Vh, int g5)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)12 * Vh) return;
    const double s = (g5 && (int)(t / Vh) >= 6) ? -1.0 : 1.0;  // spins 2, 3
    const double2 u = x2[t], v = x1[t], w = x0[t];
    y[t] = make_double2(s * (a * u.x + b * v.x + c * w.x), s * (a * u.y + b * v.y + c * w.y));
}

// ---------------------------------------------------------------------------
// deterministic two-stage sums of squares
// ---------------------------------------------------------------------------
constexpr int RED_BLOCKS = 512;

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

__global__ void k_sumsq_part(const double* x, int64_t n, double* part)
{
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        acc += x[k] * x[k];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sum_final(const double* part, int n, double* out, double scale)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += part[k];
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = scale * acc;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
// c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), key bumped by the Weyl
// constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ double u53(unsigned a, unsigned b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

// the two normals of counter index q
__device__ __forceinline__ double2 normal_pair(uint64_t q, uint2 key, unsigned stream, unsigned traj)
{
    const uint4 w = philox(make_uint4((unsigned)q, (unsigned)(q >> 32), stream, traj), key);
    const double u1 = u53(w.x, w.y), u2 = u53(w.z, w.w);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    return make_double2(rad * cs, rad * sn);
}

__global__ void k_normals(double* out, int64_t n, uint2 key, unsigned stream, unsigned traj, double scale)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * q >= n) return;
    const double2 v = normal_pair((uint64_t)q, key, stream, traj);
    out[2 * q] = scale * v.x;
    if (2 * q + 1 < n) out[2 * q + 1] = scale * v.y;
}

// complex Gaussian spinor (density exp(-|eta|^2)) written straight into the
// internal layout; component (s, c) of the ABI field uses counter s*12 + c
__global__ void k_normal_spinor(double2* full, int Vh, uint2 key, unsigned stream, unsigned traj)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)24 * Vh) return;
    const int par = (int)(t / (12 * (int64_t)Vh));
    const int comp = (int)((t / Vh) % 12);
    const int i = (int)(t % Vh);
    const int64_t site = (int64_t)par * Vh + i;
    const double2 v = normal_pair((uint64_t)(site * 12 + comp), key, stream, traj);
    const double r = 0.70710678118654752440;
    full[t] = make_double2(r * v.x, r * v.y);
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
#define LAUNCH_CHECK(h)                                                               \
    do {                                                                              \
        (h)->launches += 1;                                                           \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess) {                                                      \
            (h)->err = std::string("kernel launch: ") + cudaGetErrorString(e_);       \
            return LQCD_ERR_CUDA;                                                     \
        }                                                                             \
    } while (0)

int pack_spinor(lqcd_ctx* h, double2* dst, const double* abi, int par0, int npar)
{
    const int Vh = h->g.Vh;
    cudaEvent_t ev;
    prof_begin(h, 4, &ev);
    k_pack_spinor<<<nblk((int64_t)npar * Vh), BS, 0, h->stream>>>(dst, (const double2*)abi, Vh, par0, npar);
    LAUNCH_CHECK(h);
    prof_end(h, 4, ev, 2.0 * 192.0 * npar * Vh);
    return LQCD_OK;
}

int unpack_spinor(lqcd_ctx* h, double* abi, const double2* src, int par0, int npar)
{
    const int Vh = h->g.Vh;
    cudaEvent_t ev;
    prof_begin(h, 4, &ev);
    k_unpack_spinor<<<nblk((int64_t)npar * Vh), BS, 0, h->stream>>>((double2*)abi, src, Vh, par0, npar);
    LAUNCH_CHECK(h);
    prof_end(h, 4, ev, 2.0 * 192.0 * npar * Vh);
    return LQCD_OK;
}

int convert_spinor(lqcd_ctx* h, SpinorF dst, int dprec, SpinorF src, int sprec, int n)
{
    const int nb = nblk(n);
#define CV(a, b) \
    if (sprec == a && dprec == b) k_convert<a, b><<<nb, BS, 0, h->stream>>>(dst, src, n)
    CV(PREC64, PREC32); else CV(PREC64, PREC16); else CV(PREC32, PREC64); else CV(PREC16, PREC64);
    else CV(PREC64, PREC64); else CV(PREC32, PREC32); else CV(PREC16, PREC16); else CV(PREC32, PREC16);
    else CV(PREC16, PREC32); else CV(PREC64, PRECBF); else CV(PRECBF, PREC64); else CV(PRECBF, PRECBF);
    else CV(PREC32, PRECBF); else CV(PRECBF, PREC32);
    else {
        h->err = "convert_spinor: unsupported precision pair";
        return LQCD_ERR_ARG;
    }
#undef CV
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int pack_gauge(lqcd_ctx* h, const double* abi)
{
    const int Vh = h->g.Vh;
    k_pack_gauge<<<nblk((int64_t)8 * Vh), BS, 0, h->stream>>>(h->U64, h->U32, h->U16, (const double2*)abi, Vh);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int refresh_low_precision(lqcd_ctx* h)
{
    const int Vh = h->g.Vh;
    k_refresh_low<<<nblk((int64_t)8 * Vh), BS, 0, h->stream>>>(h->U64, h->U32, h->U16, Vh);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int unpack_gauge(lqcd_ctx* h, double* abi)
{
    const int Vh = h->g.Vh;
    k_unpack_gauge<<<nblk((int64_t)8 * Vh), BS, 0, h->stream>>>((double2*)abi, h->U64, Vh);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int index_maps(lqcd_ctx* h, int32_t* maps)
{
    k_index_maps<<<nblk(h->g.V), BS, 0, h->stream>>>(maps, h->g);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int embed_boundary(lqcd_ctx* h, double2* full, const double* coords, int nface)
{
    LQ_CUDA(h, cudaMemsetAsync(full, 0, sizeof(double2) * 24 * (size_t)h->g.Vh, h->stream));
    k_embed<<<nblk((h->g.nb / 2) * h->g.V3), BS, 0, h->stream>>>(full, (const double2*)coords, h->g, nface);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int project_boundary(lqcd_ctx* h, double* coords, const double2* full, int nface)
{
    k_project<<<nblk((h->g.nb / 2) * nface * h->g.V3), BS, 0, h->stream>>>((double2*)coords, full, h->g, nface);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int axpby_full(lqcd_ctx* h, double2* y, double a, const double2* x, double b, int colour)
{
    cudaEvent_t ev;
    prof_begin(h, 4, &ev);
    k_axpby<<<nblk((int64_t)24 * h->g.Vh), BS, 0, h->stream>>>(y, a, x, b, h->g, colour);
    LAUNCH_CHECK(h);
    prof_end(h, 4, ev, 3.0 * 384.0 * h->g.Vh);
    return LQCD_OK;
}

int keep_colour(lqcd_ctx* h, double2* y, int colour)
{
    return axpby_full(h, y, 0.0, nullptr, 1.0, colour);
}

int gamma5_full(lqcd_ctx* h, double2* y, const double2* x)
{
    k_gamma5<<<nblk((int64_t)24 * h->g.Vh), BS, 0, h->stream>>>(y, x, h->g.Vh);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int lincomb_even(lqcd_ctx* h, double2* y, double a, const double2* x1, double b, const double2* x0, int g5)
{
    k_lincomb_even<<<nblk((int64_t)12 * h->g.Vh), BS, 0, h->stream>>>(y, a, x1, b, x0, h->g.Vh, g5);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int lincomb3_even(lqcd_ctx* h, double2* y, double a, const double2* x2, double b, const double2* x1, double c,
                  const double2* x0, int g5)
{
    k_lincomb3_even<<<nblk((int64_t)12 * h->g.Vh), BS, 0, h->stream>>>(y, a, x2, b, x1, c, x0, h->g.Vh, g5);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int norm2_dev(lqcd_ctx* h, const double* x, int64_t n, double* dev_out)
{
    k_sumsq_part<<<RED_BLOCKS, BS, 0, h->stream>>>(x, n, h->red_part);
    k_sum_final<<<1, 1024, 0, h->stream>>>(h->red_part, RED_BLOCKS, dev_out, 1.0);
    h->launches += 1;
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int rng_normals(lqcd_ctx* h, double* out, int64_t n, uint64_t seed, uint32_t stream, uint32_t traj,
                double scale)
{
    if (n <= 0) return LQCD_OK;
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    k_normals<<<nblk((n + 1) / 2), BS, 0, h->stream>>>(out, n, key, stream, traj, scale);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int rng_spinor(lqcd_ctx* h, double2* full, uint64_t seed, uint32_t stream, uint32_t traj)
{
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    k_normal_spinor<<<nblk((int64_t)24 * h->g.Vh), BS, 0, h->stream>>>(full, h->g.Vh, key, stream, traj);
    LAUNCH_CHECK(h);
    return LQCD_OK;
}

int read_scalars(lqcd_ctx* h, int n, double* host)
{
    LQ_CUDA(h, cudaMemcpyAsync(h->red_host, h->red_out, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    LQ_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < n; ++k) host[k] = h->red_host[k];
    return LQCD_OK;
}

int reduction_blocks() { return RED_BLOCKS; }
