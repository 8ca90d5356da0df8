// Host harness for the boundary-closure extension map of the box kernels
// (ew_bc_dev.cuh, compiled for the host): prints, for every face code, short
// and longer axes and points far outside them, the active index and sign the
// map returns ("code n p index sign"; index -1 = a Dirichlet wall, value 0),
// once with 32-bit and once with 64-bit indices.
#include <cstdint>
#include <cstdio>

#include "ew_bc_dev.cuh"

using namespace ew;

int main() {
    for (int code = 0; code < 4; ++code) {
        const int nn = (code & 1) + ((code >> 1) & 1);
        for (int n = 1 + nn; n <= 12; ++n) {
            for (int p = -4 * n - 20; p <= 5 * n + 20; ++p) {
                int s32 = 0;
                const int i32 = ext_axis<int>(p, n, code, s32);
                int s64 = 0;
                const int64_t i64 = ext_axis<int64_t>((int64_t)p, (int64_t)n, code, s64);
                if (i32 < 0) s32 = 0;
                if (i64 < 0) s64 = 0;
                printf("%d %d %d %d %d %lld %d\n", code, n, p, i32, s32, (long long)i64, s64);
            }
        }
    }
    return 0;
}
