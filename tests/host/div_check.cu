// Host check of the multiply-high division by invariant integers that the
// cell-coordinate decomposition uses (Granlund and Montgomery, Sec. 4):
// div_magic(n, m, sh) == n / d for every divisor d in [1, 8192] on the
// multiples of d and their neighbours and on seeded random n, for large
// divisors on a dense sweep, and the (x, y, z) of a cell index for lattice
// shapes that are not powers of two.  Prints "ok" and exits 0 on success.
#include <cstdio>
#include <cstdint>

#include "../../paper_1904_02108_gb300/csrc/common.cuh"

using namespace lbmibm;

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint32_t next_u32() {  // SplitMix64, upper half
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return (uint32_t)((z ^ (z >> 31)) >> 32);
}

int main() {
  long bad = 0;
  for (uint32_t d = 1; d <= 8192; d++) {
    uint32_t m;
    int sh;
    divisor_magic(d, m, sh);
    auto chk = [&](uint32_t n) {
      if (div_magic(n, m, sh) != n / d && bad++ < 5) printf("d=%u n=%u\n", d, n);
    };
    for (uint64_t k = 0; k < 2000; k++) {
      const uint64_t b = k * d;
      if (b > 0xffffffffull) break;
      chk((uint32_t)b);
      if (b) chk((uint32_t)(b - 1));
      if (b + 1 <= 0xffffffffull) chk((uint32_t)(b + 1));
    }
    for (int k = 0; k < 500; k++) chk(next_u32());
    chk(0xffffffffu);
    chk(0x7fffffffu);
  }
  const uint32_t big[] = {12288u, 100000u, 1000003u, 1u << 20, (1u << 31) - 1u, 1u << 31};
  for (uint32_t d : big) {
    uint32_t m;
    int sh;
    divisor_magic(d, m, sh);
    for (uint64_t n = 0; n <= 0xffffffffull; n += 65521)
      if (div_magic((uint32_t)n, m, sh) != (uint32_t)n / d && bad++ < 5)
        printf("d=%u n=%llu\n", d, (unsigned long long)n);
  }
  // cell coordinates n = (z ny + y) nx + x of whole lattices
  const int shapes[][3] = {{44, 40, 48}, {36, 20, 12}, {384, 384, 384}, {160, 160, 320}, {12, 20, 36}};
  for (const auto &s : shapes) {
    Geometry g{};
    g.nx = s[0];
    g.ny = s[1];
    g.nz = s[2];
    geometry_divisors(g);
    const uint32_t nc = (uint32_t)s[0] * s[1] * s[2];
    const uint32_t step = nc > 4000000u ? 7u : 1u;
    for (uint32_t n = 0; n < nc; n += step) {
      const uint32_t r = div_magic(n, g.mx, g.shx);
      const uint32_t x = n - r * (uint32_t)g.nx, z = div_magic(r, g.my, g.shy);
      const uint32_t y = r - z * (uint32_t)g.ny;
      if ((x != n % g.nx || y != (n / g.nx) % g.ny || z != n / (g.nx * g.ny)) && bad++ < 5)
        printf("shape %d %d %d n=%u\n", s[0], s[1], s[2], n);
    }
  }
  if (bad) {
    printf("%ld mismatches\n", bad);
    return 1;
  }
  printf("ok\n");
  return 0;
}
