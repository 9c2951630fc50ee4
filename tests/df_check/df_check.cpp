// Host check of the double-float arithmetic of the double sweeps of the
// mixed-precision path, against long-double arithmetic.  Prints the
// largest relative errors seen; the pytest driver checks them.
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "lqcd_df.cuh"

static uint64_t st = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64()
{  // splitmix64
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double uni() { return (double)(next_u64() >> 11) * 0x1.0p-53; }
// |x| log-uniform in [2^lo, 2^hi), random sign
static double rnd(int lo, int hi)
{
    const double m = 1.0 + uni();
    const int e = lo + (int)(uni() * (hi - lo));
    return ((next_u64() & 1) ? -1.0 : 1.0) * ldexp(m, e);
}
static long double val(df a) { return (long double)a.hi + (long double)a.lo; }

int main()
{
    long double e_split = 0, e_add = 0, e_mul = 0, e_dot = 0, e_chain = 0, e_back = 0, lo_ulp = 0;
    int bad_special = 0;
    for (int n = 0; n < 200000; ++n) {
        const double x = rnd(-70, 70), y = rnd(-70, 70);
        const df a = df_split(x), b = df_split(y);
        e_split = fmaxl(e_split, fabsl(val(a) - x) / fabsl((long double)x));
        lo_ulp = fmaxl(lo_ulp, fabsl((long double)a.lo) / ldexpl(1.0L, ilogbl(a.hi) - 23));
        // a sum with cancellation: error relative to |x| + |y|
        const double y2 = (n & 1) ? -x * (1.0 + rnd(-30, -1)) : y;
        const df b2 = df_split(y2);
        const long double s = val(a) + val(b2);
        e_add = fmaxl(e_add, fabsl(val(a + b2) - s) / (fabsl(val(a)) + fabsl(val(b2))));
        // products inside the float range (the sweeps' values are O(1e-12 .. 1e4))
        const df a3 = df_split(rnd(-40, 40)), b3 = df_split(rnd(-40, 40));
        const long double p = val(a3) * val(b3);
        e_mul = fmaxl(e_mul, fabsl(val(a3 * b3) - p) / fabsl(p));
        e_back = fmaxl(e_back, fabsl((long double)df_to_double(a) - val(a)) / fabsl(val(a)));
        // a complex 3-vector product row as in the link multiplication
        double u[6], v[6];
        for (int k = 0; k < 6; ++k) {
            u[k] = rnd(-3, 1);
            v[k] = rnd(-6, 4);
        }
        df re(0), im(0);
        long double rr = 0, ri = 0, mag = 0;
        for (int k = 0; k < 3; ++k) {
            const df ur = df_split(u[2 * k]), ui = df_split(u[2 * k + 1]);
            const df vr = df_split(v[2 * k]), vi = df_split(v[2 * k + 1]);
            re = re + (ur * vr - ui * vi);
            im = im + (ur * vi + ui * vr);
            rr += val(ur) * val(vr) - val(ui) * val(vi);
            ri += val(ur) * val(vi) + val(ui) * val(vr);
            mag += fabsl(val(ur) * val(vr)) + fabsl(val(ui) * val(vi)) + fabsl(val(ur) * val(vi)) +
                   fabsl(val(ui) * val(vr));
        }
        e_dot = fmaxl(e_dot, fmaxl(fabsl(val(re) - rr), fabsl(val(im) - ri)) / mag);
        // a long unnormalised chain: 48 products summed (one output
        // component of a hopping sweep), relative to the sum of |terms|
        df acc(0);
        long double ex = 0, mg = 0;
        for (int k = 0; k < 48; ++k) {
            const df p = df_split(rnd(-3, 1)), q = df_split(rnd(-6, 4));
            acc = ((k & 3) == 1) ? acc - p * q : acc + p * q;
            ex += ((k & 3) == 1 ? -1 : 1) * val(p) * val(q);
            mg += fabsl(val(p) * val(q));
        }
        e_chain = fmaxl(e_chain, fabsl(val(acc) - ex) / mg);
        e_chain = fmaxl(e_chain, fabsl(val(df_norm(acc)) - val(acc)) / mg);
    }
    // zeros, a power of two, huge and tiny values
    if (val(df_split(0.0)) != 0 || val(df_split(-0.0)) != 0) ++bad_special;
    if (val(df_split(0.75)) != 0.75L || df_split(0.75).lo != 0.f) ++bad_special;
    if (!isinf(df_split(1e300).hi)) ++bad_special;
    if (!isnan(df_split(NAN).hi)) ++bad_special;
    if (fabsl(val(df_split(1e-20)) - 1e-20L) > 1e-20L * 0x1.0p-46L) ++bad_special;
    if (fabsl(val(df_split(3e-30)) - 3e-30L) > 3e-30L * 0x1.0p-23L) ++bad_special;  // below 2^-80: hi only
    if (val(df_split(1e-300)) != 0 && fabsl(val(df_split(1e-300))) > 1e-299L) ++bad_special;
    printf("split %.3Le\nadd %.3Le\nmul %.3Le\ndot %.3Le\nchain %.3Le\nback %.3Le\nlo_ulp %.3Lf\nspecial %d\n",
           e_split, e_add, e_mul, e_dot, e_chain, e_back, lo_ulp, bad_special);
    return 0;
}
