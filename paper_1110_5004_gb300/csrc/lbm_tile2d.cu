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
// S0 keeps the pulled f of the tile's own cells and S2 their pulled gbar for S3, which splits
// each cell's collision between two threads (f and gbar).
// Every per-cell operation is the shared stage function the row march uses (lbm_device.cuh), with
// the same neighbour values: cells next to a wall also write their value into the mirrored ghost
// position, as in the row march, so the state is bitwise the one the row march computes.
// Scope: s by Eq. 5 (s_form 0) and the mu-term order-parameter equilibrium (f_form 0), any storage
// and boundaries; other configurations run the row march.
#include <vector>

#include "lbm_internal.h"

namespace lbm {

template <int TX, int TY>
struct Smem2D {
  static constexpr int FW = TX + 6, FH = TY + 6;   // frame: the tile and a 3-cell halo
  float hi[FH][FW], lo[FH][FW], mu[FH][FW], p[FH][FW], ux[FH][FW], uy[FH][FW];
  float rec[10][TY][TX];   // S2 -> S3 record of the tile's cells (Rec fields phi .. ogr3)
  float gb[Q][TY][TX];     // their pulled gbar populations
  unsigned int f3[Q - 1][TY][TX];   // their pulled f_1..f_8 (stored bits), handed from S0 to S3
};

// One step of tile `tile` (row-major over tiles_x columns of tiles) from g.src into g.dst.  COH:
// population loads through L2 only, for a launch in which other CTAs write the state it reads.
// XW, YW: walls possible on x, on y; false (a periodic axis) compiles out that axis's wall tests
// and ghost writes.
template <int ST, int TX, int TY, int NT, bool COH, bool XW = true, bool YW = true>
__device__ __forceinline__ void tile2d_step(const Phys& P, const Grid& g, int tiles_x, int tile, Smem2D<TX, TY>& sm) {
  using S = Smem2D<TX, TY>;
  constexpr int FW = S::FW, FH = S::FH;
  const int t = threadIdx.x;
  const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
  const bool xwall = XW && g.bc_x == BC_WALL, ywall = YW && g.bc_y == BC_WALL;

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
    if constexpr (!XW) cn.wl = cn.wr = false;
    if constexpr (!YW) rn.wb = rn.wt = false;
  };
  // Every population load of this thread is issued first, all at once: f of its S0 cells and
  // gbar of its S2 cells; the passes then wait on the loads they use.
  constexpr int C0 = (FW * FH + NT - 1) / NT, C2 = ((FW - 4) * (FH - 4) + NT - 1) / NT;
  // Two threads per tile cell in S3: a cell's f collision goes to thread k and its gbar collision
  // to thread k + TX * TY, so the longest stage runs at half the chain.
  static_assert(NT >= 2 * TX * TY, "S3 needs two threads per tile cell");
  unsigned int f0raw[C0][NF], g2raw[C2][Q];
#pragma unroll
  for (int c = 0; c < C0; ++c) {
    const int k = t + c * NT, i = k % FW, j = k / FW, x = x0 - 3 + i, y = y0 - 3 + j;
    if (k < FW * FH && real(x, y)) {
      ColNb cn;
      RowNb rn;
      nbr(x, y, cn, rn);
      gather9<ST, 0, COH>(g.src, cn, rn, f0raw[c]);
      f0raw[c][Q] = ST == ST_FP32 ? ld_raw<ST, COH>(g.src, PLANE_F0LO, cell_at(rn.b0, cn.c0)) : 0u;
    }
  }
#pragma unroll
  for (int c = 0; c < C2; ++c) {
    const int k = t + c * NT, i = 2 + k % (FW - 4), j = 2 + k / (FW - 4), x = x0 - 3 + i, y = y0 - 3 + j;
    if (k < (FW - 4) * (FH - 4) && real(x, y)) {
      ColNb cn;
      RowNb rn;
      nbr(x, y, cn, rn);
      gather9<ST, Q, COH>(g.src, cn, rn, g2raw[c]);
    }
  }

  // ---- S0: phi on the frame; the pulled f_1..f_8 of the tile's own cells are kept for S3
#pragma unroll
  for (int c = 0; c < C0; ++c) {
    const int k = t + c * NT, i = k % FW, j = k / FW, x = x0 - 3 + i, y = y0 - 3 + j;
    if (k >= FW * FH || !real(x, y)) continue;
    float fp[NF];
#pragma unroll
    for (int a = 0; a < Q; ++a) fp[a] = dec_pop<ST>(f0raw[c][a], a);
    fp[Q] = __uint_as_float(f0raw[c][Q]);
    float hi, lo;
    phi_pair<ST>(fp, g.isf, hi, lo);
    put(sm.hi, i, j, x, y, hi);
    put(sm.lo, i, j, x, y, lo);
    const int ti = i - 3, tj = j - 3;
    if (ti >= 0 && ti < TX && tj >= 0 && tj < TY) {
#pragma unroll
      for (int a = 1; a < Q; ++a) sm.f3[a - 1][tj][ti] = f0raw[c][a];
    }
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
    for (int a = 0; a < Q; ++a) gb[a] = dec_pop<ST>(g2raw[c][a], Q + a);
    const S2Out s2 = s2_cell<ST>(P, ph, gphx, gphy, gmx, gmy, sm.mu[j][i], sdef, gb, g.isg);
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
  {
    const int k = t % (TX * TY), ti = k % TX, tj = k / TX, i = ti + 3, j = tj + 3, x = x0 + ti, y = y0 + tj;
    if (t < 2 * TX * TY && x < g.nx && y < g.ny) {
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
      float f[Q], gb[Q];
      const CellB cell = cell_at(y * g.row_bytes, col_bytes<ST>(x));
      if (t < TX * TY) {   // f: needs phi div u and the phi pair, not p
        const float phiD = P.ch_conv ? phi_div_u(r.phi, &sm.ux[j - 1][i], &sm.ux[j][i], &sm.ux[j + 1][i],
                                                 &sm.uy[j - 1][i], &sm.uy[j + 1][i])
                                     : 0.0f;
        f[0] = 0.0f;   // unused: f_0 follows from the phi pair
#pragma unroll
        for (int a = 1; a < Q; ++a) f[a] = dec_pop<ST>(sm.f3[a - 1][tj][ti], a);
#pragma unroll
        for (int a = 0; a < Q; ++a) gb[a] = 0.0f;   // unused by the f collision
        collide_store<ST, false, COLLIDE_F>(P, r, 0.0f, 0.0f, 0.0f, sm.hi[j][i], sm.lo[j][i], phiD, f, gb, g, cell);
      } else {              // gbar: needs p and grad p
        float gpx, gpy;
        grad12(&sm.p[j - 1][i], &sm.p[j][i], &sm.p[j + 1][i], gpx, gpy);
#pragma unroll
        for (int a = 0; a < Q; ++a) f[a] = 0.0f;    // unused by the gbar collision
#pragma unroll
        for (int a = 0; a < Q; ++a) gb[a] = sm.gb[a][tj][ti];
        collide_store<ST, false, COLLIDE_G>(P, r, sm.p[j][i], gpx, gpy, 0.0f, 0.0f, 0.0f, f, gb, g, cell);
      }
    }
  }
}

template <int ST, int TX, int TY, int NT, bool XW, bool YW>
__global__ void __launch_bounds__(NT) k_tile2d(Phys P, Grid g, int tiles_x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // Launched as a programmatic dependent of the previous step: wait until that grid has
  // completed and its stores are visible, then let the next step's grid be scheduled, so that
  // its launch overlaps this one instead of following it.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  tile2d_step<ST, TX, TY, NT, false, XW, YW>(P, g, tiles_x, blockIdx.x, *reinterpret_cast<Smem2D<TX, TY>*>(smem_raw));
}

// Shared memory to ask for so that at most `cap` CTAs fit on an SM (at least `need`): a grid of
// few tiles then spreads evenly over the SMs instead of piling several CTAs onto some while
// others idle.  0 when the device attributes cannot be read.
static int smem_for_cap(int need, int cap) {
  struct Attrs {
    int per_sm = 0, reserved = 0, optin = 0;
  };
  // read once per process (one GPU per process), thread-safely: host threads may step
  // simulations concurrently
  static const Attrs at = [] {
    Attrs a;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&a.per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&a.reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&a.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      a = Attrs{};
    }
    return a;
  }();
  if (at.per_sm <= 0) return need;
  const int want = (at.per_sm / (cap + 1) - at.reserved + 16 + 15) / 16 * 16;   // cap + 1 no longer fit
  if (want <= need || want > at.optin || cap * (want + at.reserved) > at.per_sm) return need;
  return want;
}

template <int ST, int TX, int TY, int NT, bool XW, bool YW>
static cudaError_t launch_tile2d_shape(const Phys& P, const Grid& g, int sms, cudaStream_t st) {
  using S = Smem2D<TX, TY>;
  static bool attr_set = false;   // one GPU per process
  if (!attr_set) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tile2d<ST, TX, TY, NT, XW, YW>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int tx = (g.nx + TX - 1) / TX, ty = (g.ny + TY - 1) / TY;
  const int tiles = tx * ty, cap = (tiles + sms - 1) / sms;   // CTAs per SM for one even wave
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem_for_cap((int)sizeof(S), cap);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tile2d<ST, TX, TY, NT, XW, YW>, P, g, tx);
}

constexpr int T2D_TX = 16, T2D_TY = 8, T2D_NT = 256, T2D_NT_WAVE = 384;

// The wall forms: both axes periodic, walls on y only (the paper's experiments), or general.
template <int ST, int NT>
static cudaError_t launch_tile2d_bc(const Phys& P, const Grid& g, int sms, cudaStream_t st) {
  if (g.bc_x != BC_WALL && g.bc_y != BC_WALL) return launch_tile2d_shape<ST, T2D_TX, T2D_TY, NT, false, false>(P, g, sms, st);
  if (g.bc_x != BC_WALL) return launch_tile2d_shape<ST, T2D_TX, T2D_TY, NT, false, true>(P, g, sms, st);
  return launch_tile2d_shape<ST, T2D_TX, T2D_TY, NT, true, true>(P, g, sms, st);
}

// 16 x 8 cells per CTA.  256 threads: every frame cell of S0 in two rounds, one for S1 and S2,
// and the collisions split between the f and gbar threads.  Measured against 16 x 8 / 128
// threads, 16 x 4 / 256, 8 x 8 / 64, 128 and 256, 16 x 16 / 256, 32 x 4 / 256 and 32 x 8 / 256
// on 128^2, 300 x 150, 150 x 450, 256 x 1024 and 512^2 grids: fastest or within 3 % on each.
// 384 threads (S0 in one round; 3 CTAs per SM) is 10-12 % faster on grids whose tiles fit one
// wave of it (128^2, 300 x 150) and 9-18 % slower on the others, so it runs where the tiles fit
// one wave; 512 threads was slower than 384 on every grid.  Either way at most ceil(tiles / SMs)
// CTAs share an SM (smem_for_cap).

template <int ST>
static cudaError_t launch_tile2d_st(const Phys& P, const Grid& g, int sms, cudaStream_t st) {
  static int slots = -1;   // CTAs of the 384-thread form resident at once (one GPU per process)
  if (slots < 0) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, k_tile2d<ST, T2D_TX, T2D_TY, T2D_NT_WAVE, true, true>, T2D_NT_WAVE, sizeof(Smem2D<T2D_TX, T2D_TY>));
    if (e != cudaSuccess) return e;
    slots = occ * sms;
  }
  const long long tiles = (long long)((g.nx + T2D_TX - 1) / T2D_TX) * ((g.ny + T2D_TY - 1) / T2D_TY);
  if (tiles <= slots) return launch_tile2d_bc<ST, T2D_NT_WAVE>(P, g, sms, st);
  return launch_tile2d_bc<ST, T2D_NT>(P, g, sms, st);
}

// ---- Resident form: one launch advances n steps.  Every CTA stays on the device and steps its
// tiles (tile = blockIdx.x, + gridDim.x, ...); before a step a tile waits only until the tiles
// within its reach have finished the previous step, which also means they have read what the
// step overwrites.  A step of a tile reads cells up to REACH away in x and y (the 3-cell halo of
// S0 and the pull), so its reach is the tiles owning a cell of the tile grown by REACH.  The
// waits cannot deadlock: a CTA takes its tiles in order, step by step, so the unfinished tile of
// the lowest step always has every tile it waits for done.  Every wait is bounded: after
// timeout_ns it raises the status word and the launch ends.
constexpr int REACH = 4;
constexpr int NB_MAX = 16;   // a tile grown by 4 meets at most 4 x 4 tiles of 16 x 8 (a ragged one included)

struct Resident {
  unsigned int* flags;    // per tile: base + steps it has finished in this launch
  unsigned int* status;   // 0, or RES_GAVE_UP after a wait ran out (cleared by the host)
  const int* reach;       // per tile NB_MAX tile indices within reach, itself excluded, -1 padded
  unsigned int base;      // flag value of every tile when the launch starts
  int nsteps, ntiles;
  long long timeout_ns;
  int hold_tile;          // this tile never announces a finished step (-1: none)
};
constexpr unsigned int RES_GAVE_UP = 1u;

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait until every tile within reach of `tile` has finished `need` steps of this launch; lane i
// of warp 0 watches neighbour i.  False (in every thread) when the launch gives up.
__device__ __forceinline__ bool wait_reach(const Resident& R, int tile, int need) {
  bool quit = false;
  if (threadIdx.x < NB_MAX) {
    const int n = __ldg(R.reach + tile * NB_MAX + threadIdx.x);
    if (n >= 0) {
      const unsigned int* f = R.flags + n;
      const unsigned int want = R.base + (unsigned int)need;
      if ((int)(ld_acquire(f) - want) < 0) {
        const unsigned long long t0 = global_ns();
        for (;;) {
          __nanosleep(32);
          if ((int)(ld_acquire(f) - want) >= 0) break;
          if (ld_acquire(R.status) != 0u) {   // another tile gave up: so does this launch
            quit = true;
            break;
          }
          if (global_ns() - t0 > (unsigned long long)R.timeout_ns) {
            atomicCAS(R.status, 0u, RES_GAVE_UP);
            quit = true;
            break;
          }
        }
      }
    }
  }
  return !__syncthreads_or(quit);
}

template <int ST, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_tile2d_resident(Phys P, Grid g, int tiles_x, Resident R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem2D<TX, TY>& sm = *reinterpret_cast<Smem2D<TX, TY>*>(smem_raw);
  // a launch that gave up leaves the state undefined: later launches do nothing until the host
  // has read the status and reset it
  if (__syncthreads_or(threadIdx.x == 0 && ld_acquire(R.status) != 0u)) return;
  Grid h = g;   // odd steps run back from dst into src
  h.src = g.dst;
  h.dst = const_cast<void*>(g.src);
  for (int s = 0; s < R.nsteps; ++s) {
    for (int tile = blockIdx.x; tile < R.ntiles; tile += gridDim.x) {
      if (s > 0 && !wait_reach(R, tile, s)) return;
      tile2d_step<ST, TX, TY, NT, true>(P, (s & 1) ? h : g, tiles_x, tile, sm);
      __syncthreads();   // every store of the tile issued (and shared memory free for the next)
      if (threadIdx.x == 0 && tile != R.hold_tile) {
        __threadfence();
        st_release(R.flags + tile, R.base + (unsigned int)(s + 1));
      }
    }
  }
}

// Tiles within reach of each tile (itself excluded), NB_MAX per tile, -1 padded.
static bool reach_table(const Grid& g, int tx_n, int ty_n, int* out) {
  for (int ty = 0; ty < ty_n; ++ty)
    for (int tx = 0; tx < tx_n; ++tx) {
      int xs[NB_MAX], ys[NB_MAX], nxs = 0, nys = 0;
      const int x0 = tx * T2D_TX, x1 = (x0 + T2D_TX < g.nx ? x0 + T2D_TX : g.nx) - 1;
      const int y0 = ty * T2D_TY, y1 = (y0 + T2D_TY < g.ny ? y0 + T2D_TY : g.ny) - 1;
      for (int c = x0 - REACH; c <= x1 + REACH; ++c) {
        if (g.bc_x == BC_WALL && (c < 0 || c >= g.nx)) continue;
        const int k = ((c % g.nx) + g.nx) % g.nx / T2D_TX;
        bool seen = false;
        for (int i = 0; i < nxs; ++i) seen |= xs[i] == k;
        if (!seen) {
          if (nxs == NB_MAX) return false;
          xs[nxs++] = k;
        }
      }
      for (int c = y0 - REACH; c <= y1 + REACH; ++c) {
        if (g.bc_y == BC_WALL && (c < 0 || c >= g.ny)) continue;
        const int k = ((c % g.ny) + g.ny) % g.ny / T2D_TY;
        bool seen = false;
        for (int i = 0; i < nys; ++i) seen |= ys[i] == k;
        if (!seen) {
          if (nys == NB_MAX) return false;
          ys[nys++] = k;
        }
      }
      int* row = out + (size_t)(ty * tx_n + tx) * NB_MAX;
      int n = 0;
      for (int i = 0; i < NB_MAX; ++i) row[i] = -1;
      for (int j = 0; j < nys; ++j)
        for (int i = 0; i < nxs; ++i) {
          const int k = ys[j] * tx_n + xs[i];
          if (k == ty * tx_n + tx) continue;
          if (n == NB_MAX) return false;
          row[n++] = k;
        }
    }
  return true;
}

template <int ST>
static cudaError_t launch_resident_st(lbm_sim* s, const Grid& g, int n) {
  using S = Smem2D<T2D_TX, T2D_TY>;
  auto* k = k_tile2d_resident<ST, T2D_TX, T2D_TY, T2D_NT>;
  static int occ = 0;   // one GPU per process
  if (occ == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(S));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, T2D_NT, sizeof(S));
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
  }
  const int tx = (g.nx + T2D_TX - 1) / T2D_TX, ty = (g.ny + T2D_TY - 1) / T2D_TY, nt = tx * ty;
  const int slots = occ * s->sms;
  Resident R{};
  R.flags = s->res_mem;
  R.status = s->res_mem + nt;
  R.reach = reinterpret_cast<const int*>(s->res_mem + nt + 1);
  R.base = s->res_base;
  R.nsteps = n;
  R.ntiles = nt;
  R.timeout_ns = s->res_timeout_ns;
  R.hold_tile = s->res_hold;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nt < slots ? nt : slots);
  cfg.blockDim = dim3(T2D_NT);
  cfg.dynamicSmemBytes = sizeof(S);
  cfg.stream = s->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident at once: the waits need it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, s->phys, g, tx, R);
}

bool tile2d_eligible(const lbm_params& p) { return p.s_form == 0 && p.f_form == 0; }

int resident_tiles(int nx, int ny) {
  return ((nx + T2D_TX - 1) / T2D_TX) * ((ny + T2D_TY - 1) / T2D_TY);
}

// Flags, status word and reach table of the simulation, allocated on first use and zeroed.
cudaError_t resident_prepare(lbm_sim* s) {
  if (s->res_mem) return cudaSuccess;
  const int nt = resident_tiles(s->nx, s->ny);
  const size_t words = (size_t)nt + 1 + (size_t)nt * NB_MAX;
  std::vector<int> host((size_t)nt * NB_MAX);
  const Grid g = make_grid(s, nullptr, nullptr);
  if (!reach_table(g, (s->nx + T2D_TX - 1) / T2D_TX, (s->ny + T2D_TY - 1) / T2D_TY, host.data()))
    return cudaErrorInvalidValue;   // cannot happen for 16 x 8 tiles and a reach of 4
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, words * sizeof(unsigned int), s->stream);
  if (e != cudaSuccess) return e;
  s->res_mem = static_cast<unsigned int*>(p);
  e = cudaMemsetAsync(s->res_mem, 0, ((size_t)nt + 1) * sizeof(unsigned int), s->stream);
  if (e == cudaSuccess)   // pageable source: staged before the call returns
    e = cudaMemcpyAsync(s->res_mem + nt + 1, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  s->res_base = 0;
  return e;
}

// Zero the flags and the status word (after a launch gave up, or a new initial state).
cudaError_t resident_reset(lbm_sim* s) {
  s->res_base = 0;
  if (!s->res_mem) return cudaSuccess;
  return cudaMemsetAsync(s->res_mem, 0, ((size_t)resident_tiles(s->nx, s->ny) + 1) * sizeof(unsigned int), s->stream);
}

cudaError_t launch_resident(lbm_sim* s, const Grid& g, int n) {
  cudaError_t e = resident_prepare(s);
  if (e != cudaSuccess) return e;
  switch (g.storage) {
    case ST_FP16: e = launch_resident_st<ST_FP16>(s, g, n); break;
    case ST_BF16: e = launch_resident_st<ST_BF16>(s, g, n); break;
    default: e = launch_resident_st<ST_FP32>(s, g, n); break;
  }
  if (e == cudaSuccess) {
    s->res_base += (unsigned int)n;
    s->res_used = true;
  }
  return e;
}

cudaError_t launch_tile2d(const Phys& P, const Grid& g, int sms, cudaStream_t st) {
  switch (g.storage) {
    case ST_FP16: return launch_tile2d_st<ST_FP16>(P, g, sms, st);
    case ST_BF16: return launch_tile2d_st<ST_BF16>(P, g, sms, st);
    default: return launch_tile2d_st<ST_FP32>(P, g, sms, st);
  }
}

}  // namespace lbm
