// Host harness for the double-FP32 pair arithmetic (ew_dd.cuh, compiled for
// the host): prints the largest error of each operation over random operands,
// measured in long double, relative to the operand magnitudes.
#include <cmath>
#include <cstdio>
#include <random>

#include "ew_dd.cuh"

using namespace ew;

static long double val(dd x) { return (long double)x.hi + (long double)x.lo; }

int main() {
    std::mt19937_64 rng(20250718);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    double conv = 0, add = 0, mul = 0, fma = 0, canc = 0, nonoverlap = 0;
    for (int i = 0; i < 1000000; ++i) {
        const double a = U(rng) * std::ldexp(1.0, (int)(U(rng) * 20));
        const double b = U(rng) * std::ldexp(1.0, (int)(U(rng) * 20));
        const dd x(a), y(b), w(U(rng));
        const long double xa = val(x), ya = val(y), wa = val(w);
        conv = std::fmax(conv, (double)(std::fabs(val(x) - (long double)a) / std::fabs((long double)a)));
        const dd s = x + y, p = x * y, f = dd_fma(x, y, w);
        add = std::fmax(add, (double)(std::fabs(val(s) - (xa + ya)) / (std::fabs(xa) + std::fabs(ya))));
        mul = std::fmax(mul, (double)(std::fabs(val(p) - xa * ya) / std::fabs(xa * ya)));
        fma = std::fmax(fma, (double)(std::fabs(val(f) - (xa * ya + wa)) / (std::fabs(xa * ya) + std::fabs(wa))));
        const dd z(-a * (1.0 + 1e-9 * U(rng)));
        const dd c = x + z;
        canc = std::fmax(canc, (double)(std::fabs(val(c) - (xa + val(z))) / (std::fabs(xa) + std::fabs(val(z)))));
        // renormalised results: |lo| <= ulp(hi) / 2
        for (dd r : {s, p, f})
            if (r.hi != 0.0f)
                nonoverlap = std::fmax(nonoverlap, (double)(std::fabs(r.lo) / (0.5 * std::fabs(std::nextafter(r.hi, 2 * r.hi) - r.hi))));
    }
    std::printf("%.6e %.6e %.6e %.6e %.6e %.6e\n", conv, add, mul, fma, canc, nonoverlap);
    return 0;
}
