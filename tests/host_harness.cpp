// Test harness for the library's host-side geometry helpers (lbm_host.cu):
// reads a uint8 [ny][nx] mask from a file and prints, one per line,
//   solids <count> <sum of indices> <first> <last>   (solid_nodes, threaded for large masks)
//   solids1 <count> <sum of indices>                 (the same scan with no threads: row chunks of one)
//   cv <x0> <x1> <y0> <y1>                           (auto_cv)
//   base <lb_x> <lb_y> <fb_x> <fb_y>                 (base_sums over that box, rho0 = 1, %.17g)
//   base_own <lb_x> <lb_y> <fb_x> <fb_y>             (the same without the shared solid list)
// Usage: host_harness <mask file> <nx> <ny> <periodic>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "lbm_host.h"

int main(int argc, char **argv)
{
    if (argc != 5) return 2;
    const int nx = std::atoi(argv[2]), ny = std::atoi(argv[3]), periodic = std::atoi(argv[4]);
    std::vector<uint8_t> m((size_t)nx * ny);
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 3;
    const size_t got = std::fread(m.data(), 1, m.size(), f);
    std::fclose(f);
    if (got != m.size()) return 4;

    const std::vector<long long> s = gblbm::solid_nodes(m.data(), nx, ny);
    long long sum = 0;
    for (long long k : s) sum += k;
    std::printf("solids %zu %lld %lld %lld\n", s.size(), sum, s.empty() ? -1LL : s.front(),
                s.empty() ? -1LL : s.back());
    // one row at a time: each call is below the threading threshold
    long long n1 = 0, sum1 = 0;
    for (int y = 0; y < ny; ++y)
        for (long long k : gblbm::solid_nodes(m.data() + (size_t)y * nx, nx, 1)) {
            ++n1;
            sum1 += k + (long long)y * nx;
        }
    std::printf("solids1 %lld %lld\n", n1, sum1);

    int cv[4];
    gblbm::auto_cv(m.data(), nx, ny, periodic, cv, &s);
    std::printf("cv %d %d %d %d\n", cv[0], cv[1], cv[2], cv[3]);
    double lb[2], fb[2];
    gblbm::base_sums(m.data(), nx, ny, periodic, cv, 1.0, lb, fb, &s);
    std::printf("base %.17g %.17g %.17g %.17g\n", lb[0], lb[1], fb[0], fb[1]);
    gblbm::base_sums(m.data(), nx, ny, periodic, cv, 1.0, lb, fb, nullptr);
    std::printf("base_own %.17g %.17g %.17g %.17g\n", lb[0], lb[1], fb[0], fb[1]);
    return 0;
}
