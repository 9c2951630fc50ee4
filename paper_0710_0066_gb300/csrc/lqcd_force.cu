// lqcd_force.cu -- link forces, gauge action, link update and x0 shift.
//
// Pseudo-fermion forces.  For a link U_mu(x) moved along T^a,
// delta U = i w T^a U, and the derivative of 2 Re <a, H b> is
//   2 Re[ a(x)^dag (1-g_mu) iT^a U b(x+mu) + a(x+mu)^dag (1+g_mu) (iT^a U)^dag b(x) ]
// = -2 Im tr(T^a Y),   Y = U X1 - X2 U^dag,
//   X1 = sum_i h_i[(1-g_mu) b(x+mu)] h_i[(1-g_mu) a(x)]^dag,
//   X2 = sum_i h_i[(1+g_mu) b(x)]   h_i[(1+g_mu) a(x+mu)]^dag,
// with h the two-spin upper half of the projected spinor (the lower half is
// a unitary image of it, so the four-spin trace equals the two-spin one).
// All of this runs in double precision on the double solution vectors.
#include <math.h>

#include "lqcd_common.cuh"

namespace {

constexpr int BS = 128;
constexpr double INV_SQRT3 = 0.57735026918962576451;

__device__ __forceinline__ void site_at(const Geo& g, const int x[4], int& par, int& i)
{
    par = (x[0] + x[1] + x[2] + x[3]) & 1;
    i = lex_of(g, x) >> 1;
}

__device__ __forceinline__ void shifted(const Geo& g, const int x[4], int mu, int d, int y[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) y[k] = x[k];
    y[mu] += d;
    if (y[mu] >= g.L[mu]) y[mu] -= g.L[mu];
    if (y[mu] < 0) y[mu] += g.L[mu];
}

// 2 Im tr(T^a Y) for the eight Gell-Mann generators T^a = lambda^a / 2
template <class T>
__device__ __forceinline__ void lie_im2(const Su3<T>& Y, double f[8])
{
    f[0] = (double)(Y.m[1][0].im + Y.m[0][1].im);
    f[1] = (double)(Y.m[0][1].re - Y.m[1][0].re);
    f[2] = (double)(Y.m[0][0].im - Y.m[1][1].im);
    f[3] = (double)(Y.m[2][0].im + Y.m[0][2].im);
    f[4] = (double)(Y.m[0][2].re - Y.m[2][0].re);
    f[5] = (double)(Y.m[2][1].im + Y.m[1][2].im);
    f[6] = (double)(Y.m[1][2].re - Y.m[2][1].re);
    f[7] = (double)(Y.m[0][0].im + Y.m[1][1].im - T(2) * Y.m[2][2].im) * INV_SQRT3;
}

template <class T>
__device__ __forceinline__ void su3_mul(const Su3<T>& a, const Su3<T>& b, Su3<T>& c)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j] + a.m[i][2] * b.m[2][j];
}
// c = a b^dag
template <class T>
__device__ __forceinline__ void su3_mul_nd(const Su3<T>& a, const Su3<T>& b, Su3<T>& c)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.m[i][j] = a.m[i][0] * conjx(b.m[j][0]) + a.m[i][1] * conjx(b.m[j][1]) + a.m[i][2] * conjx(b.m[j][2]);
}

template <class T>
__device__ __forceinline__ void outer_acc(const HalfSp<T>& hb, const HalfSp<T>& ha, Su3<T>& X)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            X.m[i][j] = X.m[i][j] + hb.c[0][i] * conjx(ha.c[0][j]) + hb.c[1][i] * conjx(ha.c[1][j]);
}

struct BilTerm {
    SpinorF a[2], b[2];  // parity views of the full double fields
    int mask;
    double coef;
    int on;
};

template <class T>
__device__ __forceinline__ void load_as(const SpinorF& f, int i, Spinor<T>& s)
{
    Spinor<double> d;
    load_spinor<PREC64>(f, i, d);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) s.c[a][c] = mk((T)d.c[a][c].re, (T)d.c[a][c].im);
}

// one term for the link (x, mu) in the arithmetic of link precision PL
template <int PL>
__device__ __forceinline__ void bilinear_link(const Geo& g, const GaugeF& U, const BilTerm& T, int mu, int par,
                                              int i, const int x[4], double f[8])
{
    typedef typename Real<PL>::T R;
    if (mu == 0 ? !t_hop_kept(g, T.mask, x[0] + 1) : (T.mask == MODE_CROSS || T.mask == MODE_CROSS2)) return;
    const bool wrap = (x[mu] == g.L[mu] - 1);
    int y[4], py, iy;
    shifted(g, x, mu, +1, y);
    site_at(g, y, py, iy);
    HalfSp<R> hax, hby, hay, hbx;
    {
        Spinor<R> s;
        load_as(T.a[par], i, s);
        project(mu, -1, s, hax);
        load_as(T.b[par], i, s);
        project(mu, +1, s, hbx);
        load_as(T.a[py], iy, s);
        project(mu, +1, s, hay);
        load_as(T.b[py], iy, s);
        project(mu, -1, s, hby);
    }
    Su3<R> X1, X2, u, Y, t1, t2;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) X1.m[r][c] = X2.m[r][c] = mk(R(0), R(0));
    outer_acc(hby, hax, X1);
    outer_acc(hbx, hay, X2);
    load_link<PL>(U, mu, par, i, u);
    su3_mul(u, X1, t1);
    su3_mul_nd(X2, u, t2);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Y.m[r][c] = t1.m[r][c] - t2.m[r][c];
    double l[8];
    lie_im2(Y, l);
    const double ph = (mu == 0 && wrap && g.bc_t < 0) ? -1.0 : 1.0;
    const double s = -T.coef * ph;
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] += s * l[k];
}

// step-size factor of link (x, mu) (Sec. 2); 1 without a table
__device__ __forceinline__ double link_scale(const Geo& g, const double* ss, int mu, int x0)
{
    return ss ? ss[(mu == 0 ? g.L[0] : 0) + x0] : 1.0;
}

// F[mu][site][a] += sum over the (up to two) terms; one thread per link
template <int PL>
__global__ void __launch_bounds__(BS) k_bilinear(Geo g, GaugeF U, double* F, BilTerm T1, BilTerm T2, const double* ss)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * g.V) return;
    const int mu = t / g.V, s = t - mu * g.V;
    const int par = s >= g.Vh ? 1 : 0, i = s - par * g.Vh;
    int x[4];
    eo_coords(g, par, i, x);
    const double sc = link_scale(g, ss, mu, x[0]);
    if (sc == 0.0) return;
    double f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = 0.0;
    if (T1.on) bilinear_link<PL>(g, U, T1, mu, par, i, x, f);
    if (T2.on) bilinear_link<PL>(g, U, T2, mu, par, i, x, f);
    double4* d4 = (double4*)(F + ((size_t)mu * g.V + s) * 8);
    double4 a = d4[0], b = d4[1];
    a.x += sc * f[0]; a.y += sc * f[1]; a.z += sc * f[2]; a.w += sc * f[3];
    b.x += sc * f[4]; b.y += sc * f[5]; b.z += sc * f[6]; b.w += sc * f[7];
    d4[0] = a;
    d4[1] = b;
}

// staple sum A with U_mu(x) A the sum of the six plaquettes through the link
template <int P>
__device__ void staple(const Geo& g, const GaugeF& U, const int x[4], int mu, Su3<typename Real<P>::T>& A)
{
    typedef typename Real<P>::T R;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) A.m[r][c] = mk(R(0), R(0));
    int xm[4];
    shifted(g, x, mu, +1, xm);
#pragma unroll 1
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        int y[4], p, i;
        Su3<R> a, b, c, t, s;
        // up: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        site_at(g, xm, p, i);
        load_link<P>(U, nu, p, i, a);
        shifted(g, x, nu, +1, y);
        site_at(g, y, p, i);
        load_link<P>(U, mu, p, i, b);
        site_at(g, x, p, i);
        load_link<P>(U, nu, p, i, c);
        su3_mul_nd(a, b, t);
        su3_mul_nd(t, c, s);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) A.m[r][q] = A.m[r][q] + s.m[r][q];
        // down: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
        shifted(g, xm, nu, -1, y);
        site_at(g, y, p, i);
        load_link<P>(U, nu, p, i, a);
        shifted(g, x, nu, -1, y);
        site_at(g, y, p, i);
        load_link<P>(U, mu, p, i, b);
        load_link<P>(U, nu, p, i, c);
        // t = a^dag b^dag = (b a)^dag
        su3_mul(b, a, s);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) t.m[r][q] = conjx(s.m[q][r]);
        su3_mul(t, c, s);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) A.m[r][q] = A.m[r][q] + s.m[r][q];
    }
}

// F += coef * dS_G/dw^a,  dS_G/dw^a = -beta/3 Re tr(i T^a U A) = beta/6 * 2 Im tr(T^a U A)
template <int P>
__global__ void __launch_bounds__(BS) k_gauge_force(Geo g, GaugeF U, double* F, double c, const double* ss)
{
    typedef typename Real<P>::T R;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * g.V) return;
    const int mu = t / g.V, s = t - mu * g.V;
    const int par = s >= g.Vh ? 1 : 0, i = s - par * g.Vh;
    int x[4];
    eo_coords(g, par, i, x);
    c *= link_scale(g, ss, mu, x[0]);
    if (c == 0.0) return;
    Su3<R> A, u, Y;
    staple<P>(g, U, x, mu, A);
    load_link<P>(U, mu, par, i, u);
    su3_mul(u, A, Y);
    double l[8];
    lie_im2(Y, l);
    double* d = F + ((size_t)mu * g.V + s) * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] += c * l[k];
}

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

// partial sums of Re tr of the six plaquettes at each site
__global__ void k_plaq_part(Geo g, GaugeF U, double* part)
{
    double acc = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
        const int par = s >= g.Vh ? 1 : 0, i = s - par * g.Vh;
        int x[4];
        eo_coords(g, par, i, x);
        for (int mu = 1; mu < 4; ++mu)
            for (int nu = 0; nu < mu; ++nu) {
                int y[4], p, j;
                Su3<double> a, b, c, d, t, r;
                load_link<PREC64>(U, mu, par, i, a);
                shifted(g, x, mu, +1, y);
                site_at(g, y, p, j);
                load_link<PREC64>(U, nu, p, j, b);
                shifted(g, x, nu, +1, y);
                site_at(g, y, p, j);
                load_link<PREC64>(U, mu, p, j, c);
                load_link<PREC64>(U, nu, par, i, d);
                su3_mul(a, b, t);
                su3_mul_nd(t, c, r);
                su3_mul_nd(r, d, t);
                acc += t.m[0][0].re + t.m[1][1].re + t.m[2][2].re;
            }
    }
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

// average force per time slice (the diagnostic of Sec. 3, Fig. 1): block
// x0 sums |F| = (sum_a F_a^2)^(1/2) over the slice's space-like links (out[x0])
// and its time-like links (out[L0 + x0]) in a fixed order
__global__ void k_force_profile(Geo g, const double* F, double* out)
{
    const int x0 = blockIdx.x;
    double sp = 0.0, tm = 0.0;
    for (int l3 = threadIdx.x; l3 < g.V3; l3 += blockDim.x) {
        const int lex = x0 * g.V3 + l3;
        int x[4];
        x[3] = l3 % g.L[3];
        x[2] = (l3 / g.L[3]) % g.L[2];
        x[1] = l3 / (g.L[3] * g.L[2]);
        x[0] = x0;
        const int s = ((x[0] + x[1] + x[2] + x[3]) & 1) * g.Vh + (lex >> 1);
        for (int mu = 0; mu < 4; ++mu) {
            const double* f = F + ((size_t)mu * g.V + s) * 8;
            double n = 0.0;
#pragma unroll
            for (int a = 0; a < 8; ++a) n += f[a] * f[a];
            if (mu == 0) tm += sqrt(n);
            else sp += sqrt(n);
        }
    }
    sp = block_sum(sp);
    tm = block_sum(tm);
    if (threadIdx.x == 0) {
        out[x0] = sp / (3.0 * g.V3);
        out[g.L[0] + x0] = tm / g.V3;
    }
}

// exp(iQ) for traceless hermitian Q by the Cayley-Hamilton form
// exp(iQ) = f0 + f1 Q + f2 Q^2 (Morningstar & Peardon, PRD 69 (2004) 054501).
// For the molecular dynamics' small steps (c1 = tr Q^2 / 2 <= 1) the
// coefficients come from the Taylor series of exp(iQ) reduced by
// Cayley-Hamilton, Q^3 = c1 Q + c0 (c0 = det Q): with Q^n = a0 + a1 Q + a2 Q^2,
// Q^(n+1) = c0 a2 + (a0 + c1 a2) Q + a1 Q^2, and f_j = sum_n i^n a_j / n!,
// a scalar recurrence without transcendental functions (terms fall below
// 1e-17 of the leading ones after about 6 + 3 |Q| steps); larger Q use the
// closed form with the trigonometric functions.
// 1 / n!, n = 0..40, for the series of expiq (constant memory: every
// thread of a warp reads the same entry)
constexpr double inv_factorial(int n) { return n <= 1 ? 1.0 : inv_factorial(n - 1) / n; }
__constant__ double c_invfact[41] = {
    inv_factorial(0),  inv_factorial(1),  inv_factorial(2),  inv_factorial(3),  inv_factorial(4),  inv_factorial(5),
    inv_factorial(6),  inv_factorial(7),  inv_factorial(8),  inv_factorial(9),  inv_factorial(10), inv_factorial(11),
    inv_factorial(12), inv_factorial(13), inv_factorial(14), inv_factorial(15), inv_factorial(16), inv_factorial(17),
    inv_factorial(18), inv_factorial(19), inv_factorial(20), inv_factorial(21), inv_factorial(22), inv_factorial(23),
    inv_factorial(24), inv_factorial(25), inv_factorial(26), inv_factorial(27), inv_factorial(28), inv_factorial(29),
    inv_factorial(30), inv_factorial(31), inv_factorial(32), inv_factorial(33), inv_factorial(34), inv_factorial(35),
    inv_factorial(36), inv_factorial(37), inv_factorial(38), inv_factorial(39), inv_factorial(40)};

// Q^2 of a hermitian Q from its six distinct entries (real diagonal)
__device__ __forceinline__ void herm_square(const Su3<double>& Q, Su3<double>& Q2)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double d = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) d += Q.m[i][k].re * Q.m[i][k].re + Q.m[i][k].im * Q.m[i][k].im;
        Q2.m[i][i] = mk(d, 0.0);
#pragma unroll
        for (int j = i + 1; j < 3; ++j) {
            const cx<double> v = Q.m[i][0] * Q.m[0][j] + Q.m[i][1] * Q.m[1][j] + Q.m[i][2] * Q.m[2][j];
            Q2.m[i][j] = v;
            Q2.m[j][i] = conjx(v);
        }
    }
}

__device__ void expiq(const Su3<double>& Q, Su3<double>& E)
{
    Su3<double> Q2;
    herm_square(Q, Q2);
    const double c1 = 0.5 * (Q2.m[0][0].re + Q2.m[1][1].re + Q2.m[2][2].re);
    cx<double> f0, f1, f2;
    if (c1 >= 1e-12 && c1 <= 1.0) {
        const cx<double> det = Q.m[0][0] * (Q.m[1][1] * Q.m[2][2] - Q.m[1][2] * Q.m[2][1]) -
                               Q.m[0][1] * (Q.m[1][0] * Q.m[2][2] - Q.m[1][2] * Q.m[2][0]) +
                               Q.m[0][2] * (Q.m[1][0] * Q.m[2][1] - Q.m[1][1] * Q.m[2][0]);
        const double c0 = det.re;
        double a0 = 1.0, a1 = 0.0, a2 = 0.0;  // Q^n coordinates
        double r0 = 1.0, r1 = 0.0, r2 = 0.0, i0 = 0.0, i1 = 0.0, i2 = 0.0;
        const double qn = sqrt(2.0 * c1);  // Frobenius norm of Q: |Q^n| <= qn^n
        double qp = 1.0;                    // qn^n
        for (int n = 1; n <= 40; ++n) {
            const double b0 = c0 * a2, b1 = a0 + c1 * a2, b2 = a1;
            a0 = b0;
            a1 = b1;
            a2 = b2;
            const double w = c_invfact[n];
            qp *= qn;
            const double bound = qp * w;
            // i^n: 1, i, -1, -i
            switch (n & 3) {
                case 0: r0 += w * a0; r1 += w * a1; r2 += w * a2; break;
                case 1: i0 += w * a0; i1 += w * a1; i2 += w * a2; break;
                case 2: r0 -= w * a0; r1 -= w * a1; r2 -= w * a2; break;
                default: i0 -= w * a0; i1 -= w * a1; i2 -= w * a2; break;
            }
            if (bound < 1e-18) break;
        }
        f0 = mk(r0, i0);
        f1 = mk(r1, i1);
        f2 = mk(r2, i2);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cx<double> v = f1 * Q.m[r][c] + f2 * Q2.m[r][c];
                if (r == c) v = v + f0;
                E.m[r][c] = v;
            }
        return;
    }
    if (c1 < 1e-12) {
        // |Q| < 1.5e-6: series to fourth order
        Su3<double> Q3, Q4;
        su3_mul(Q2, Q, Q3);
        su3_mul(Q2, Q2, Q4);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cx<double> v = mul_i(Q.m[r][c]) - 0.5 * Q2.m[r][c] - (1.0 / 6.0) * mul_i(Q3.m[r][c]) +
                               (1.0 / 24.0) * Q4.m[r][c];
                if (r == c) v.re += 1.0;
                E.m[r][c] = v;
            }
        return;
    }
    // c0 = det Q (real)
    const cx<double> det = Q.m[0][0] * (Q.m[1][1] * Q.m[2][2] - Q.m[1][2] * Q.m[2][1]) -
                           Q.m[0][1] * (Q.m[1][0] * Q.m[2][2] - Q.m[1][2] * Q.m[2][0]) +
                           Q.m[0][2] * (Q.m[1][0] * Q.m[2][1] - Q.m[1][1] * Q.m[2][0]);
    const double c0 = det.re;
    const double c0a = fabs(c0);
    const double c0max = 2.0 * pow(c1 / 3.0, 1.5);
    const double ratio = fmin(1.0, c0a / c0max);
    const double theta = acos(ratio);
    const double u = sqrt(c1 / 3.0) * cos(theta / 3.0);
    const double w = sqrt(c1) * sin(theta / 3.0);
    const double u2 = u * u, w2 = w * w;
    double xi0;
    if (fabs(w) < 0.05)
        xi0 = 1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0));
    else
        xi0 = sin(w) / w;
    double s2u, c2u, su, cu;
    sincos(2.0 * u, &s2u, &c2u);
    sincos(u, &su, &cu);
    const double cw = cos(w);
    const cx<double> e2 = mk(c2u, s2u), em = mk(cu, -su);
    const cx<double> h0 = (u2 - w2) * e2 + em * mk(8.0 * u2 * cw, 2.0 * u * (3.0 * u2 + w2) * xi0);
    const cx<double> h1 = (2.0 * u) * e2 - em * mk(2.0 * u * cw, -(3.0 * u2 - w2) * xi0);
    const cx<double> h2 = e2 - em * mk(cw, 3.0 * u * xi0);
    const double dinv = 1.0 / (9.0 * u2 - w2);
    f0 = dinv * h0;
    f1 = dinv * h1;
    f2 = dinv * h2;
    if (c0 < 0.0) {  // f_j(-c0) = (-1)^j conj(f_j(c0))
        f0 = conjx(f0);
        f1 = -conjx(f1);
        f2 = conjx(f2);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<double> v = f1 * Q.m[r][c] + f2 * Q2.m[r][c];
            if (r == c) v = v + f0;
            E.m[r][c] = v;
        }
}

__device__ void reunitarise(Su3<double>& u)
{
    double n0 = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) n0 += u.m[0][j].re * u.m[0][j].re + u.m[0][j].im * u.m[0][j].im;
    n0 = rsqrt(n0);
#pragma unroll
    for (int j = 0; j < 3; ++j) u.m[0][j] = n0 * u.m[0][j];
    cx<double> d = mk(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 3; ++j) d = d + cjmul(u.m[0][j], u.m[1][j]);
#pragma unroll
    for (int j = 0; j < 3; ++j) u.m[1][j] = u.m[1][j] - d * u.m[0][j];
    double n1 = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) n1 += u.m[1][j].re * u.m[1][j].re + u.m[1][j].im * u.m[1][j].im;
    n1 = rsqrt(n1);
#pragma unroll
    for (int j = 0; j < 3; ++j) u.m[1][j] = n1 * u.m[1][j];
    complete_row2(u);
}

__device__ void store_link_all(double2* U64, float4* U32, uint2* U16, int Vh, int mp, int i, const Su3<double>& u)
{
    double2* d64 = U64 + (size_t)mp * 9 * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) d64[(size_t)k * Vh + i] = make_double2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const cx<double> x = u.m[(2 * k) / 3][(2 * k) % 3], y = u.m[(2 * k + 1) / 3][(2 * k + 1) % 3];
        store_low_link_word(U32, U16, Vh, mp, k, i, x.re, x.im, y.re, y.im);
    }
}

// U_mu(x) <- exp(i dt P_mu(x)) U_mu(x), P = sum_a p^a T^a; all three copies
__global__ void __launch_bounds__(BS) k_update(Geo g, double2* U64, float4* U32, uint2* U16, const double* P, double dt,
                                              const double* ss)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * g.V) return;
    const int mu = t / g.V, s = t - mu * g.V;
    const int par = s >= g.Vh ? 1 : 0, i = s - par * g.Vh;
    dt *= link_scale(g, ss, mu, (2 * i) / g.V3);
    if (dt == 0.0) return;  // a frozen link
    const double* p = P + ((size_t)mu * g.V + s) * 8;
    double q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = dt * p[k];
    Su3<double> Q, E, u, n;
    const double r3 = q[7] * INV_SQRT3;
    Q.m[0][0] = mk(0.5 * (q[2] + r3), 0.0);
    Q.m[1][1] = mk(0.5 * (-q[2] + r3), 0.0);
    Q.m[2][2] = mk(-r3, 0.0);
    Q.m[0][1] = mk(0.5 * q[0], -0.5 * q[1]);
    Q.m[1][0] = mk(0.5 * q[0], 0.5 * q[1]);
    Q.m[0][2] = mk(0.5 * q[3], -0.5 * q[4]);
    Q.m[2][0] = mk(0.5 * q[3], 0.5 * q[4]);
    Q.m[1][2] = mk(0.5 * q[5], -0.5 * q[6]);
    Q.m[2][1] = mk(0.5 * q[5], 0.5 * q[6]);
    expiq(Q, E);
    GaugeF G;
    G.v = U64;
    G.Vh = g.Vh;
    load_link<PREC64>(G, mu, par, i, u);
    su3_mul(E, u, n);
    reunitarise(n);
    store_link_all(U64, U32, U16, g.Vh, mu * 2 + par, i, n);
}

// U'_mu(x) = U_mu(x - shift 0hat)
__global__ void k_roll(Geo g, double2* U64, float4* U32, uint2* U16, const double2* src, int shift)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * g.V) return;
    const int mu = t / g.V, s = t - mu * g.V;
    const int par = s >= g.Vh ? 1 : 0, i = s - par * g.Vh;
    int x[4], y[4], p, j;
    eo_coords(g, par, i, x);
    shifted(g, x, 0, -shift, y);
    site_at(g, y, p, j);
    GaugeF G;
    G.v = src;
    G.Vh = g.Vh;
    Su3<double> u;
    load_link<PREC64>(G, mu, p, j, u);
    store_link_all(U64, U32, U16, g.Vh, mu * 2 + par, i, u);
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
static int launch_err(lqcd_ctx* h, const char* what)
{
    h->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->err = std::string(what) + ": " + cudaGetErrorString(e);
        return LQCD_ERR_CUDA;
    }
    return LQCD_OK;
}

static BilTerm make_term(lqcd_ctx* h, const double2* a, const double2* b, int mask, double coef)
{
    BilTerm T;
    T.on = (a != nullptr && b != nullptr) ? 1 : 0;
    for (int p = 0; p < 2; ++p) {
        T.a[p] = sp64((double2*)a, p, h->g.Vh);
        T.b[p] = sp64((double2*)b, p, h->g.Vh);
    }
    T.mask = mask;
    T.coef = coef;
    return T;
}

int force_bilinear(lqcd_ctx* h, double* F, const double2* a1, const double2* b1, int mask1, double coef1,
                   const double2* a2, const double2* b2, int mask2, double coef2, int prec, const double* ss)
{
    BilTerm T1 = make_term(h, a1, b1, mask1, coef1), T2 = make_term(h, a2, b2, mask2, coef2);
    cudaEvent_t ev;
    prof_begin(h, 2, &ev);
    const int nb = (4 * h->g.V + BS - 1) / BS;
    if (prec == PREC64)
        k_bilinear<PREC64><<<nb, BS, 0, h->stream>>>(h->g, gauge_view(h, PREC64), F, T1, T2, ss);
    else
        k_bilinear<PREC32><<<nb, BS, 0, h->stream>>>(h->g, gauge_view(h, PREC32), F, T1, T2, ss);
    LQ_TRY(launch_err(h, "force kernel"));
    const int nt = T1.on + T2.on;
    // per site: two spinors of each term, four links, F read and written
    prof_end(h, 2, ev, (double)h->g.V * (nt * 2.0 * 192.0 + 4.0 * 144.0 + 2.0 * 256.0));
    return LQCD_OK;
}

int gauge_force_kick(lqcd_ctx* h, double* F, double coef, int prec, const double* ss)
{
    // coef * (beta/6) is folded in by the caller
    cudaEvent_t ev;
    prof_begin(h, 3, &ev);
    const int nb = (4 * h->g.V + BS - 1) / BS;
    if (prec == PREC64)
        k_gauge_force<PREC64><<<nb, BS, 0, h->stream>>>(h->g, gauge_view(h, PREC64), F, coef, ss);
    else
        k_gauge_force<PREC32><<<nb, BS, 0, h->stream>>>(h->g, gauge_view(h, PREC32), F, coef, ss);
    LQ_TRY(launch_err(h, "gauge force kernel"));
    prof_end(h, 3, ev, (double)h->g.V * (4.0 * 144.0 + 2.0 * 256.0));
    return LQCD_OK;
}

int plaquette_sum(lqcd_ctx* h, double* dev_out)
{
    const int nb = h->red_blocks;
    k_plaq_part<<<nb, 256, 0, h->stream>>>(h->g, gauge_view(h, PREC64), h->red_part);
    k_sum_final<<<1, 1024, 0, h->stream>>>(h->red_part, nb, dev_out, 1.0);
    h->launches += 1;
    return launch_err(h, "plaquette kernel");
}

int update_links(lqcd_ctx* h, const double* P, double dt, const double* ss)
{
    cudaEvent_t ev;
    prof_begin(h, 3, &ev);
    k_update<<<(4 * h->g.V + BS - 1) / BS, BS, 0, h->stream>>>(h->g, h->U64, h->U32, h->U16, P, dt, ss);
    LQ_TRY(launch_err(h, "link update kernel"));
    prof_end(h, 3, ev, (double)h->g.V * 4.0 * (2.0 * 144.0 + 64.0 + 48.0 + 24.0));
    return LQCD_OK;
}

int roll_links(lqcd_ctx* h, int shift)
{
    // src: the saved copy (caller copies the current field there first)
    k_roll<<<(4 * h->g.V + BS - 1) / BS, BS, 0, h->stream>>>(h->g, h->U64, h->U32, h->U16, h->U64_save, shift);
    return launch_err(h, "roll kernel");
}

int force_profile(lqcd_ctx* h, const double* F, double* out)
{
    k_force_profile<<<h->g.L[0], 256, 0, h->stream>>>(h->g, F, out);
    return launch_err(h, "force profile kernel");
}

int kinetic_sum(lqcd_ctx* h, const double* P, double* dev_out)
{
    return norm2_dev(h, P, (int64_t)32 * h->g.V, dev_out);
}

// ---------------------------------------------------------------------------
// Gauge action for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another
// framework owns the whole device memory pool, real-time or signal-safe host
// threads that must not trigger the implicit device synchronisation of an
// allocation, and hosts that only hand out pre-sized buffers.  They also
// cannot create an lqcd handle (lqcd_create allocates its workspace), so
// this entry point takes the gauge field directly and keeps its per-block
// partial sums in a fixed array compiled into the library.
//
// The array is a file-scope __device__ variable of 16384 doubles (128 KiB);
// every GPU that loads the library holds it until the process exits.  One
// block of 128 threads handles 128 sites, so at most 16384 * 128 =
// 2,097,152 sites (32^3 x 64) fit; larger lattices are rejected with
// LQCD_ERR_GEOM.  Every call shares the array: the used entries are fully
// rewritten by each call before they are read (nothing has to start at
// zero), and calls that overlap on the GPU (different streams, or threads
// with no ordering between them) race on it.  The device address of the
// array is looked up with cudaGetSymbolAddress on the first call on each
// device, with that device current; make that first call before any stream
// capture.  No cudaMalloc, cudaFree or other allocating routine is called.
// ---------------------------------------------------------------------------
#include <mutex>

constexpr int STATIC_SITES_PER_BLOCK = 128;
constexpr int STATIC_MAX_BLOCKS = 16384;
static __device__ __align__(256) double g_static_partials[STATIC_MAX_BLOCKS];

namespace {

__device__ __forceinline__ void abi_link(const double2* U, int V, int mu, int s, Su3<double>& u)
{
    const double2* p = U + ((size_t)mu * V + s) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) u.m[k / 3][k % 3] = mk(p[k].x, p[k].y);
}

__device__ __forceinline__ int abi_site(const Geo& g, const int x[4])
{
    return ((x[0] + x[1] + x[2] + x[3]) & 1) * g.Vh + (lex_of(g, x) >> 1);
}

// Re tr of the six plaquettes at each of this block's sites, read straight
// from the C-ABI gauge layout; one partial sum per block
__global__ void __launch_bounds__(STATIC_SITES_PER_BLOCK) k_plaq_static(Geo g, const double2* U, double* part)
{
    const int s = blockIdx.x * STATIC_SITES_PER_BLOCK + threadIdx.x;
    double acc = 0.0;
    if (s < g.V) {
        const int par = s >= g.Vh ? 1 : 0, i = s - par * g.Vh;
        int x[4];
        eo_coords(g, par, i, x);
        for (int mu = 1; mu < 4; ++mu)
            for (int nu = 0; nu < mu; ++nu) {
                int y[4];
                Su3<double> a, b, c, d, t, r;
                abi_link(U, g.V, mu, s, a);
                shifted(g, x, mu, +1, y);
                abi_link(U, g.V, nu, abi_site(g, y), b);
                shifted(g, x, nu, +1, y);
                abi_link(U, g.V, mu, abi_site(g, y), c);
                abi_link(U, g.V, nu, s, d);
                su3_mul(a, b, t);
                su3_mul_nd(t, c, r);
                su3_mul_nd(r, d, t);
                acc += t.m[0][0].re + t.m[1][1].re + t.m[2][2].re;
            }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_plaq_static_final(const double* part, int n, double* out, double beta, double inv_norm)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += part[k];
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
        out[0] = -beta / 3.0 * acc;
        out[1] = acc * inv_norm;
    }
}

std::mutex g_static_mu;
double* g_static_ptr[128] = {nullptr};

// device address of g_static_partials on the current device (looked up once)
int static_partials(double** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return LQCD_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_partials) != cudaSuccess || !p) return LQCD_ERR_CUDA;
        g_static_ptr[dev] = (double*)p;
    }
    *out = g_static_ptr[dev];
    return LQCD_OK;
}

}  // namespace

extern "C" int lqcd_gauge_action_static(const int L[4], const double* U, double beta, double* out, void* stream)
{
    if (!L || !U || !out) return LQCD_ERR_ARG;
    // every extent and every partial product stays within the site bound
    // before the next multiplication, so the volume cannot overflow
    const int64_t max_sites = (int64_t)STATIC_MAX_BLOCKS * STATIC_SITES_PER_BLOCK;
    int64_t V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (L[mu] < 2 || (L[mu] & 1) || L[mu] > max_sites) return LQCD_ERR_GEOM;
        V *= L[mu];
        if (V > max_sites) return LQCD_ERR_GEOM;
    }
    const int64_t nblocks = (V + STATIC_SITES_PER_BLOCK - 1) / STATIC_SITES_PER_BLOCK;
    double* part = nullptr;
    const int st = static_partials(&part);
    if (st != LQCD_OK) return st;
    Geo g;
    for (int mu = 0; mu < 4; ++mu) g.L[mu] = L[mu];
    g.V = (int)V;
    g.Vh = g.V / 2;
    g.V3 = L[1] * L[2] * L[3];
    g.l0 = 1;
    g.nb = L[0];
    g.bc_t = 1;
    g.Sh = g.V3 / 2;
    g.l0s = 0;
    geo_finish(g);
    cudaStream_t s = (cudaStream_t)stream;
    k_plaq_static<<<(unsigned)nblocks, STATIC_SITES_PER_BLOCK, 0, s>>>(g, (const double2*)U, part);
    k_plaq_static_final<<<1, 1024, 0, s>>>(part, (int)nblocks, out, beta, 1.0 / (18.0 * (double)V));
    return cudaGetLastError() == cudaSuccess ? LQCD_OK : LQCD_ERR_CUDA;
}
