// lbm_frame.cuh -- the opposed-jets boundary set of Sec. 4.3 on a frame of
// outside nodes.
//
// The outermost x and y layers of the grid (x = 0, nx - 1; y = 0, ny - 1) are
// frame nodes: they take no collision.  After every collision each frame node
// holds, in the AA location of its outgoing populations, the post-collision
// populations that stream into the domain:
//   * x faces, rows jet_y0 <= y < jet_y1 (the nozzles): the complete
//     equilibrium of the inlet state (the incoming populations replaced by
//     equilibria);
//   * x faces, other rows: free-slip walls, the mirror image of the boundary
//     node with the x velocity reflected (specular reflection halfway
//     between the frame node and the boundary node);
//   * y faces (the outlets): a copy of the boundary node (zero normal
//     derivative);
//   * corners: the x-face rule of the nearest boundary row.
// The receivers of those populations add the frame node's deferred terms
// (lbm_stencil.cuh), so a frame node also holds the side fields of its image:
// the gradient inputs as the nearest boundary node's values (Phi_x negated
// beyond a free-slip wall), the deferred-term fields mirrored or copied with
// its populations, and zero deferred terms at the nozzles (the equilibrium
// enters as it is).
#pragma once

#include "lbm_stencil.cuh"

namespace lbm {

// Frame node k of one z plane: the bottom row (y = 0), the top row, then the
// left and right columns of the rows between.
template <class P>
__device__ __forceinline__ void frame_node(const P& p, long long k, int& x, int& y) {
  const int nx = p.nx, ny = p.ny;
  if (k < nx) { x = (int)k; y = 0; return; }
  if (k < 2LL * nx) { x = (int)(k - nx); y = ny - 1; return; }
  const long long r = k - 2LL * nx;
  y = 1 + (int)(r / 2);
  x = (r % 2 == 0) ? 0 : nx - 1;
}
template <class P>
__host__ __device__ __forceinline__ long long frame_count(const P& p) {
  return (2LL * p.nx + 2LL * (p.ny - 2)) * p.nz;
}

// The image of frame node (x, y) in plane z: the nearest boundary node b and
// the rule (0: copy, 1: free-slip mirror in x, 2: nozzle `inlet` 0 or 1).
struct FrameImage {
  long long b;
  int rule, inlet;
};
template <class P>
__device__ __forceinline__ FrameImage frame_image(const P& p, int x, int y, int z) {
  const int xc = x < 1 ? 1 : (x > p.nx - 2 ? p.nx - 2 : x);
  const int yc = y < 1 ? 1 : (y > p.ny - 2 ? p.ny - 2 : y);
  FrameImage im;
  im.b = ((long long)z * p.ny + yc) * p.nx + xc;
  im.inlet = x == 0 ? 0 : 1;
  if (x == 0 || x == p.nx - 1) im.rule = (yc >= p.jet_y0 && yc < p.jet_y1) ? 2 : 1;
  else im.rule = 0;
  return im;
}

// Populations: after a collision of parity `parity`, every population that a
// frame node sends into the domain, written where the receiver will read it
// (the AA location of the frame node's outgoing population).  jet: the
// complete inlet equilibria [(L * 27 + i) * 2 + inlet]; base: the reference
// rest equilibria [L * 27 + i] of the stored deviations.
template <int M, class Real, class Store>
__global__ void __launch_bounds__(BLOCK_LIGHT)
frame_pops_kernel(const DevParams<Real> p, Store* __restrict__ pops, const double* __restrict__ jet,
                  const double* __restrict__ base, int parity) {
  const long long t = gtid();
  const long long per = frame_count(p) / p.nz;
  if (t >= per * p.nz) return;
  const int z = (int)(t / per);
  int x, y;
  frame_node(p, t - (long long)z * per, x, y);
  const long long N = p.N;
  const long long g = ((long long)z * p.ny + y) * p.nx + x;
  const FrameImage im = frame_image(p, x, y, z);
  const Nbr ng = make_nbr(p, g), nb = make_nbr(p, im.b);
#pragma unroll 1
  for (int i = 0; i < Q; ++i) {
    const int cx = cx_of(i), cy = cy_of(i);
    const int tx = x + cx, ty = y + cy;
    if (tx < 1 || tx > p.nx - 2 || ty < 1 || ty > p.ny - 2) continue;   // not into the domain
    long long wn, sn; int ws, ss;
    aa_write_loc<false>(parity, ng, g, i, wn, ws);
    if (im.rule == 2) {
#pragma unroll
      for (int L = 0; L < M + 2; ++L)
        codec_store<Store, double>(p, pops, (long long)(L * Q + ws) * N + wn, L,
                                   jet[(L * Q + i) * 2 + im.inlet] - base[L * Q + i]);
    } else {
      const int j = im.rule == 1 ? i - 2 * cx : i;     // x velocity reflected at a free-slip wall
      aa_write_loc<false>(parity, nb, im.b, j, sn, ss);
#pragma unroll
      for (int L = 0; L < M + 2; ++L)
        pops[(long long)(L * Q + ws) * N + wn] = pops[(long long)(L * Q + ss) * N + sn];
    }
  }
}

// Side fields of the frame nodes.  stage 0 (after the collision): the
// gradient inputs of the first stencil pass; stage 1 (after it): G for the
// second pass, and K, theta of the deferred terms; stage 2 (after the second
// pass): X of the deferred terms.
template <class Real>
__global__ void __launch_bounds__(BLOCK_LIGHT)
frame_side_kernel(const DevParams<Real> p, Real* __restrict__ side, int stage) {
  const long long t = gtid();
  const long long per = frame_count(p) / p.nz;
  if (t >= per * p.nz) return;
  const int z = (int)(t / per);
  int x, y;
  frame_node(p, t - (long long)z * per, x, y);
  const long long N = p.N;
  const long long g = ((long long)z * p.ny + y) * p.nx + x;
  const FrameImage im = frame_image(p, x, y, z);
  auto copy = [&](int plane, Real sgn) { side[plane * N + g] = sgn * side[plane * N + im.b]; };
  const Real odd = im.rule == 1 ? Real(-1) : Real(1);          // x components beyond a free-slip wall
  if (stage == 0) {
    copy(SP_PHI + 0, odd);
    copy(SP_PHI + 1, Real(1)); copy(SP_PHI + 2, Real(1));
    copy(SP_COM, Real(1)); copy(SP_CP, Real(1)); copy(SP_S, Real(1)); copy(SP_TH, Real(1));
  } else if (stage == 1) {
    copy(SP_G + 0, Real(1)); copy(SP_G + 1, Real(1)); copy(SP_G + 2, Real(1));
    const Real k = im.rule == 2 ? Real(0) : Real(1);           // nozzles: no deferred terms
    copy(SP_K + 0, k * odd); copy(SP_K + 1, k); copy(SP_K + 2, k);
    copy(SP_THR, Real(1));
  } else {
    const Real k = im.rule == 2 ? Real(0) : Real(1);
    copy(SP_X + 0, k * odd); copy(SP_X + 1, k); copy(SP_X + 2, k);
  }
}

}  // namespace lbm
