// Device helpers shared by the lattice kernels (lbm.cu) and the brick kernels
// of the immersed boundary loop (ibm.cu): cell coordinates, the pull of Eq. 4
// and the moments of Eq. 1 in deviation form.
#pragma once

#include "common.cuh"

namespace lbmibm {

// (x, y, z) of the cell with linear index n = (z ny + y) nx + x; shifts and
// masks when nx and ny are powers of two (the same for every thread), else
// the multiply-high division when the geometry carries its constants.
__device__ __forceinline__ void cell_coords(uint32_t n, const Geometry &g, int &x, int &y,
                                            int &z) {
  const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
  if ((nx & (nx - 1)) == 0 && (ny & (ny - 1)) == 0) {
    const uint32_t r = n >> (__ffs((int)nx) - 1);
    x = (int)(n & (nx - 1));
    y = (int)(r & (ny - 1));
    z = (int)(r >> (__ffs((int)ny) - 1));
    return;
  }
  if (g.mx) {
    const uint32_t r = div_magic(n, g.mx, g.shx);
    x = (int)(n - r * nx);
    z = (int)div_magic(r, g.my, g.shy);
    y = (int)(r - (uint32_t)z * ny);
    return;
  }
  const uint32_t r = n / nx;
  x = (int)(n - r * nx);
  z = (int)(r / ny);
  y = (int)(r - (uint32_t)z * ny);
}

// Pull of Eq. 4: d[i] = stored d_i at X - e_i (periodic).  PF: loads with a
// 64-byte L2 prefetch size (for the scattered 4-cell rows of the active
// bricks); STREAM: with a 256-byte one (the dense rows of the collide).
template <typename S, bool PF = false, bool STREAM = false>
__device__ __forceinline__ void pull(const S *__restrict__ f, const Geometry &g, int x, int y,
                                     int z, float d[Q]) {
  const uint32_t nx = g.nx, ny = g.ny;
  const uint32_t xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
  const uint32_t ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
  const uint32_t zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
  // source of population i is X - e_i: e = +1 reads the "minus" neighbour
  const uint32_t X[3] = {xp, (uint32_t)x, xm};  // index by e + 1 -> X - e
  const uint32_t Y[3] = {yp, (uint32_t)y, ym};
  const uint32_t Z[3] = {zp, (uint32_t)z, zm};
  const size_t N = (size_t)g.ncell;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const uint32_t src = (Z[ez(i) + 1] * ny + Y[ey(i) + 1]) * nx + X[ex(i) + 1];
    const S *q = f + (size_t)i * N + src;
    d[i] = PF ? Store<S>::ld_pf(q) : (STREAM ? Store<S>::ld_stream(q) : Store<S>::ld(q));
  }
}

// Eq. 1 in deviation form: rho - 1 = sum d_i, rho U = sum e_i d_i.
__device__ __forceinline__ void moments(const float d[Q], float &drho, float &jx, float &jy,
                                        float &jz) {
  drho = 0.f;
  jx = jy = jz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    drho += d[i];
    if (ex(i)) jx += ex(i) > 0 ? d[i] : -d[i];
    if (ey(i)) jy += ey(i) > 0 ? d[i] : -d[i];
    if (ez(i)) jz += ez(i) > 0 ? d[i] : -d[i];
  }
}

// U0 of Eq. 1 at cell (x, y, z) from the populations after the pull of Eq. 4:
// the one arithmetic every U0 pre-computation uses (so that they agree
// bitwise).
template <typename S, bool PF = false>
__device__ __forceinline__ void cell_velocity(const S *__restrict__ f, const Geometry &g, int x,
                                              int y, int z, float &ux, float &uy, float &uz) {
  float d[Q];
  pull<S, PF>(f, g, x, y, z, d);
  float drho, jx, jy, jz;
  moments(d, drho, jx, jy, jz);
  const float inv = 1.f / (1.f + drho);
  ux = jx * inv;
  uy = jy * inv;
  uz = jz * inv;
}

}  // namespace lbmibm
