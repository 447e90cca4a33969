// Small-grid form of the fused step: one CTA computes a TX x TY tile of cells in four passes over
// shared memory instead of marching a strip of rows.
//
// On a small grid the row march is latency-bound: a segment of h rows takes h + 8 dependent row
// iterations, each waiting on the last, however few rows it has.  Here a step is one round of
// population loads (all issued at once) and four short passes separated by three barriers:
//   S0  phi on the tile plus a 3-cell halo          (pull of f, bounce-back at walls)
//   S1  mu on the tile plus 2                        (Eq. 1)
//   S2  u, p on the tile plus 1                      (pull of gbar; Eq. 4, 5, 8)
//   S3  collide and store the tile                   (grad p, phi div u, both BGK collisions)
// Every per-cell operation is the shared stage function the row march uses (lbm_device.cuh), with
// the same neighbour values: cells next to a wall also write their value into the mirrored ghost
// position, as in the row march, so the state is bitwise the one the row march computes.
// Scope: s by Eq. 5 (s_form 0) and the mu-term order-parameter equilibrium (f_form 0), any storage
// and boundaries; other configurations run the row march.
#include "lbm_internal.h"

namespace lbm {

template <int TX, int TY>
struct Smem2D {
  static constexpr int FW = TX + 6, FH = TY + 6;   // frame: the tile and a 3-cell halo
  float hi[FH][FW], lo[FH][FW], mu[FH][FW], p[FH][FW], ux[FH][FW], uy[FH][FW];
  float rec[10][TY][TX];   // S2 -> S3 record of the tile's cells (Rec fields phi .. ogr3)
  float gb[Q][TY][TX];     // their pulled gbar populations
};

template <int ST, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_tile2d(Phys P, Grid g, int tiles_x) {
  using S = Smem2D<TX, TY>;
  constexpr int FW = S::FW, FH = S::FH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S& sm = *reinterpret_cast<S*>(smem_raw);
  const int t = threadIdx.x;
  const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
  const bool xwall = g.bc_x == BC_WALL, ywall = g.bc_y == BC_WALL;

  // frame position (i, j) <-> logical cell (x0 - 3 + i, y0 - 3 + j)
  auto real = [&](int x, int y) {
    return (!xwall || (x >= 0 && x < g.nx)) && (!ywall || (y >= 0 && y < g.ny));
  };
  // write v at (i, j) and at the mirrored ghost positions of a cell next to a wall (one layer)
  auto put = [&](float (*f)[FW], int i, int j, int x, int y, float v) {
    f[j][i] = v;
    const int gi = xwall ? (x == 0 ? i - 1 : (x == g.nx - 1 ? i + 1 : -1)) : -1;
    const int gj = ywall ? (y == 0 ? j - 1 : (y == g.ny - 1 ? j + 1 : -1)) : -1;
    const bool oi = gi >= 0 && gi < FW, oj = gj >= 0 && gj < FH;
    if (oi) f[j][gi] = v;
    if (oj) f[gj][i] = v;
    if (oi && oj) f[gj][gi] = v;
  };
  auto nbr = [&](int x, int y, ColNb& cn, RowNb& rn) {
    cn = make_col<ST>(wrap1(x, g.nx), g);
    rn = make_row(wrap1(y, g.ny), g);
  };
  // Launched as a programmatic dependent of the previous step: wait until that grid has
  // completed and its stores are visible, then let the next step's grid be scheduled, so that
  // its launch overlaps this one instead of following it.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  // Every population load of this thread is issued first, all at once: f of its S0 cells, gbar
  // of its S2 cells and f of its S3 cell; the passes then wait on the loads they use.
  constexpr int C0 = (FW * FH + NT - 1) / NT, C2 = ((FW - 4) * (FH - 4) + NT - 1) / NT, C3 = (TX * TY + NT - 1) / NT;
  unsigned int f0raw[C0][NF], g2raw[C2][Q], f3raw[C3][Q];
#pragma unroll
  for (int c = 0; c < C0; ++c) {
    const int k = t + c * NT, i = k % FW, j = k / FW, x = x0 - 3 + i, y = y0 - 3 + j;
    if (k < FW * FH && real(x, y)) {
      ColNb cn;
      RowNb rn;
      nbr(x, y, cn, rn);
      gather9<ST, 0>(g.src, cn, rn, f0raw[c]);
      f0raw[c][Q] = ST == ST_FP32 ? ld_raw<ST>(g.src, PLANE_F0LO, cell_at(rn.b0, cn.c0)) : 0u;
    }
  }
#pragma unroll
  for (int c = 0; c < C2; ++c) {
    const int k = t + c * NT, i = 2 + k % (FW - 4), j = 2 + k / (FW - 4), x = x0 - 3 + i, y = y0 - 3 + j;
    if (k < (FW - 4) * (FH - 4) && real(x, y)) {
      ColNb cn;
      RowNb rn;
      nbr(x, y, cn, rn);
      gather9<ST, Q>(g.src, cn, rn, g2raw[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < C3; ++c) {
    const int k = t + c * NT, x = x0 + k % TX, y = y0 + k / TX;
    if (k < TX * TY && x < g.nx && y < g.ny) {
      ColNb cn;
      RowNb rn;
      nbr(x, y, cn, rn);
      gather9<ST, 0>(g.src, cn, rn, f3raw[c]);   // the collision's f populations
    }
  }

  // ---- S0: phi on the frame
#pragma unroll
  for (int c = 0; c < C0; ++c) {
    const int k = t + c * NT, i = k % FW, j = k / FW, x = x0 - 3 + i, y = y0 - 3 + j;
    if (k >= FW * FH || !real(x, y)) continue;
    float fp[NF];
#pragma unroll
    for (int a = 0; a < Q; ++a) fp[a] = dec_pop<ST>(f0raw[c][a], a, g.isf);
    fp[Q] = __uint_as_float(f0raw[c][Q]);
    float hi, lo;
    phi_pair(fp, hi, lo);
    put(sm.hi, i, j, x, y, hi);
    put(sm.lo, i, j, x, y, lo);
  }
  __syncthreads();
  // ---- S1: mu on the frame less one ring
  for (int k = t; k < (FW - 2) * (FH - 2); k += NT) {
    const int i = 1 + k % (FW - 2), j = 1 + k / (FW - 2), x = x0 - 3 + i, y = y0 - 3 + j;
    if (!real(x, y)) continue;
    put(sm.mu, i, j, x, y,
        chem_potential(P, &sm.hi[j - 1][i], &sm.hi[j][i], &sm.hi[j + 1][i], &sm.lo[j - 1][i], &sm.lo[j][i],
                       &sm.lo[j + 1][i]));
  }
  __syncthreads();
  // ---- S2: u, p on the tile plus one ring; the record of the tile's own cells
#pragma unroll
  for (int c = 0; c < C2; ++c) {
    const int k = t + c * NT, i = 2 + k % (FW - 4), j = 2 + k / (FW - 4), x = x0 - 3 + i, y = y0 - 3 + j;
    if (k >= (FW - 4) * (FH - 4) || !real(x, y)) continue;
    const float ph = fadd(sm.hi[j][i], sm.lo[j][i]);
    float gphx, gphy, gmx, gmy;
    grad12(&sm.hi[j - 1][i], &sm.hi[j][i], &sm.hi[j + 1][i], gphx, gphy);
    grad12(&sm.mu[j - 1][i], &sm.mu[j][i], &sm.mu[j + 1][i], gmx, gmy);
    const float sdef = P.remove_Fa ? fmul(P.s_coef6, lap6_of(&sm.mu[j - 1][i], &sm.mu[j][i], &sm.mu[j + 1][i])) : 0.0f;
    float gb[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) gb[a] = dec_pop<ST>(g2raw[c][a], Q + a, g.isg);
    const S2Out s2 = s2_cell(P, ph, gphx, gphy, gmx, gmy, sm.mu[j][i], sdef, gb);
    put(sm.p, i, j, x, y, s2.p);
    if (P.ch_conv) {
      put(sm.ux, i, j, x, y, s2.ux);
      put(sm.uy, i, j, x, y, s2.uy);
    }
    const int ti = i - 3, tj = j - 3;
    if (ti >= 0 && ti < TX && tj >= 0 && tj < TY) {
      Rec r{};
      s2_record(P, s2, ph, sm.mu[j][i], sdef, r);
      const float v[10] = {r.phi, r.mu, r.ux, r.uy, r.Fx, r.Fy, r.mrx3, r.mry3, r.og, r.ogr3};
#pragma unroll
      for (int q = 0; q < 10; ++q) sm.rec[q][tj][ti] = v[q];
#pragma unroll
      for (int a = 0; a < Q; ++a) sm.gb[a][tj][ti] = gb[a];
    }
  }
  __syncthreads();
  // ---- S3: collide and store the tile's own cells
#pragma unroll
  for (int c = 0; c < C3; ++c) {
    const int k = t + c * NT, ti = k % TX, tj = k / TX, i = ti + 3, j = tj + 3, x = x0 + ti, y = y0 + tj;
    if (k >= TX * TY || x >= g.nx || y >= g.ny) continue;
    float gpx, gpy;
    grad12(&sm.p[j - 1][i], &sm.p[j][i], &sm.p[j + 1][i], gpx, gpy);
    Rec r{};
    r.phi = sm.rec[0][tj][ti];
    r.mu = sm.rec[1][tj][ti];
    r.ux = sm.rec[2][tj][ti];
    r.uy = sm.rec[3][tj][ti];
    r.Fx = sm.rec[4][tj][ti];
    r.Fy = sm.rec[5][tj][ti];
    r.mrx3 = sm.rec[6][tj][ti];
    r.mry3 = sm.rec[7][tj][ti];
    r.og = sm.rec[8][tj][ti];
    r.ogr3 = sm.rec[9][tj][ti];
    const float phiD = P.ch_conv ? phi_div_u(r.phi, &sm.ux[j - 1][i], &sm.ux[j][i], &sm.ux[j + 1][i], &sm.uy[j - 1][i],
                                             &sm.uy[j + 1][i])
                                 : 0.0f;
    float f[Q], gb[Q];
    f[0] = 0.0f;                          // unused: f_0 follows from the phi pair
#pragma unroll
    for (int a = 1; a < Q; ++a) f[a] = dec_pop<ST>(f3raw[c][a], a, g.isf);
#pragma unroll
    for (int a = 0; a < Q; ++a) gb[a] = sm.gb[a][tj][ti];
    collide_store<ST, false>(P, r, sm.p[j][i], gpx, gpy, sm.hi[j][i], sm.lo[j][i], phiD, f, gb, g,
                             cell_at(y * g.row_bytes, col_bytes<ST>(x)));
  }
}

template <int ST, int TX, int TY, int NT>
static cudaError_t launch_tile2d_shape(const Phys& P, const Grid& g, cudaStream_t st) {
  using S = Smem2D<TX, TY>;
  static bool attr_set = false;   // one GPU per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tile2d<ST, TX, TY, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(S));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int tx = (g.nx + TX - 1) / TX, ty = (g.ny + TY - 1) / TY;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tx * ty);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sizeof(S);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tile2d<ST, TX, TY, NT>, P, g, tx);
}

// 16 x 8 cells per CTA of 256 threads: every frame cell of S0 in two rounds, one for S1 and S2.
// Measured against 16 x 8 / 128 and 384 threads, 16 x 4 / 256, 8 x 8 / 64, 128 and 256,
// 16 x 16 / 256, 32 x 4 / 256 and 32 x 8 / 256 on 128^2, 300 x 150, 150 x 450, 256 x 1024 and
// 512^2 grids: fastest or within 3 % on each but 300 x 150, where 16 x 8 / 384 is 11 % faster and
// every other grid 1-20 % slower.
template <int ST>
static cudaError_t launch_tile2d_st(const Phys& P, const Grid& g, cudaStream_t st) {
  return launch_tile2d_shape<ST, 16, 8, 256>(P, g, st);
}

bool tile2d_eligible(const lbm_params& p) { return p.s_form == 0 && p.f_form == 0; }

cudaError_t launch_tile2d(const Phys& P, const Grid& g, cudaStream_t st) {
  switch (g.storage) {
    case ST_FP16: return launch_tile2d_st<ST_FP16>(P, g, st);
    case ST_BF16: return launch_tile2d_st<ST_BF16>(P, g, st);
    default: return launch_tile2d_st<ST_FP32>(P, g, st);
  }
}

}  // namespace lbm
