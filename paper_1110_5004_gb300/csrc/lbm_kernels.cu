// Kernels of the two-distribution D2Q9 multiphase LBM: fused step, moments, initial state and
// FP64 diagnostics, with their launchers.
#include <math.h>

#include "lbm_internal.h"

namespace lbm {

// ------------------------------------------------------------------ fused step / moments

template <int NT, int MODE, int ST, bool SD, bool FF, bool XW>
// Resident CTAs per SM: 8 of 64 threads or 2 of 256 (16 warps, at most 128 registers per thread),
// 3 of 128 threads (12 warps, at most 168 registers).  Given the room, the 128-thread FP32 step
// takes 148 registers instead of 128, and on the 2048 x 512 splash its whole-wave tile (20 rows,
// 442 CTAs) ran 47.1 us per step against 49.2 us for the best tile at 4 CTAs of 128 registers.
__global__ void __launch_bounds__(NT, NT == 128 ? 3 : 512 / NT) k_tiles(Phys P, Grid g, MomentOut mo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<NT>& sm = *reinterpret_cast<Smem<NT>*>(smem_raw);
  if (MODE == MODE_STEP) {
    // launched as a programmatic dependent of the previous step: wait until that grid has
    // completed and its stores are visible, then let the next step's launch proceed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  }
  const int strip = blockIdx.x % g.n_strips;
  const int seg = blockIdx.x / g.n_strips;
  run_tile<NT, MODE, ST, SD, FF, XW>(P, g, mo, strip, seg, sm);
}

static int n_tiles(const Grid& g) { return g.n_strips * ((g.ny + g.seg_h - 1) / g.seg_h); }

// Dynamic shared memory of a row-march CTA (step or moments).  The periodic-x form (XW false)
// can need fewer registers than the general form and then fit more CTAs per SM; it is held to
// the general form's count, for which the tile heights are sized (one wave) and which measured
// faster (c3 42.8 us on 128 x 20 at 3 per SM against 45.6 us on 128 x 15 at 4, when the form
// took 128 registers), by asking for just more shared memory than one more CTA would leave room
// for.
template <int NT, bool XW>
static int step_smem_bytes() {
  int smem = (int)sizeof(Smem<NT>);
  if (XW) return smem;
  int dev = 0, per_sm = 0, reserved = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
    cudaGetLastError();
    return smem;
  }
  const int occ = tile_occupancy(NT);   // CTAs per SM of the general form
  const int cap = (per_sm / (occ + 1) - reserved + 16 + 15) / 16 * 16;
  // the general form's count must still fit
  if (cap > smem && occ * (cap + reserved) <= per_sm) smem = cap;
  return smem;
}

template <int NT, int MODE, int ST, bool SD, bool FF, bool XW = true>
static cudaError_t launch_sd(const Phys& P, const Grid& g, const MomentOut& mo, cudaStream_t st) {
  static int smem = 0;   // one GPU per process
  if (smem == 0) {
    const int want = step_smem_bytes<NT, XW>();
    cudaError_t e = cudaFuncSetAttribute(k_tiles<NT, MODE, ST, SD, FF, XW>, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    if (e != cudaSuccess) return e;
    smem = want;
  }
  if (MODE != MODE_STEP) {
    k_tiles<NT, MODE, ST, SD, FF, XW><<<n_tiles(g), NT, smem, st>>>(P, g, mo);
    return cudaGetLastError();
  }
  // consecutive steps overlap their launches (programmatic dependent launch)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_tiles(g));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tiles<NT, MODE, ST, SD, FF, XW>, P, g, mo);
}

template <int NT, int MODE, int ST>
static cudaError_t launch_nt(const Phys& P, const Grid& g, const MomentOut& mo, cudaStream_t st) {
  // the forced order-parameter form changes only the step's f collision (FP32 storage only)
  if constexpr (MODE == MODE_STEP && ST == ST_FP32) {
    if (P.f_forced)
      return P.s_direct ? launch_sd<NT, MODE, ST, true, true>(P, g, mo, st)
                        : launch_sd<NT, MODE, ST, false, true>(P, g, mo, st);
  }
  if (P.s_direct) return launch_sd<NT, MODE, ST, true, false>(P, g, mo, st);
  // a periodic x axis compiles out the ghost columns and column wall tests
  if (g.bc_x != BC_WALL) return launch_sd<NT, MODE, ST, false, false, false>(P, g, mo, st);
  return launch_sd<NT, MODE, ST, false, false>(P, g, mo, st);
}

template <int MODE, int ST>
static cudaError_t launch_st(const Phys& P, const Grid& g, const MomentOut& mo, int nt, cudaStream_t st) {
  switch (nt) {
    case 64: return launch_nt<64, MODE, ST>(P, g, mo, st);
    case 128: return launch_nt<128, MODE, ST>(P, g, mo, st);
    case 256: return launch_nt<256, MODE, ST>(P, g, mo, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int MODE>
static cudaError_t launch_tiles(const Phys& P, const Grid& g, const MomentOut& mo, int nt, cudaStream_t st) {
  switch (g.storage) {
    case ST_FP32: return launch_st<MODE, ST_FP32>(P, g, mo, nt, st);
    case ST_FP16: return launch_st<MODE, ST_FP16>(P, g, mo, nt, st);
    case ST_BF16: return launch_st<MODE, ST_BF16>(P, g, mo, nt, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int NT>
static int occupancy_nt() {
  int occ = 0;
  // the dynamic shared-memory size above 48 KB is only admitted once the attribute is set
  cudaFuncSetAttribute(k_tiles<NT, MODE_STEP, ST_FP32, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(Smem<NT>));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tiles<NT, MODE_STEP, ST_FP32, false, false, true>, NT, sizeof(Smem<NT>));
  cudaGetLastError();
  return occ > 0 ? occ : 1;
}

int tile_occupancy(int nt) {
  switch (nt) {
    case 64: return occupancy_nt<64>();
    case 256: return occupancy_nt<256>();
    default: return occupancy_nt<128>();
  }
}

cudaError_t launch_step(const Phys& P, const Grid& g, int nt, cudaStream_t st) {
  return launch_tiles<MODE_STEP>(P, g, MomentOut{}, nt, st);
}

cudaError_t launch_moments(const Phys& P, const Grid& g, const MomentOut& mo, int nt, cudaStream_t st) {
  return launch_tiles<MODE_MOMENTS>(P, g, mo, nt, st);
}

// ------------------------------------------------------------------ initial state
// fields: [0] phi0, [1] (unused), [2] ux0, [3] uy0, [4] p0 -- pitched planes; mu0 is evaluated
// where it is used.

// Post-collision-layout state whose pull gives f = f^eq(phi0, mu0, u0), gbar = g^eq(p0, rho0, u0):
// plane a at cell z holds the equilibrium of direction a at z + e_a, or, when that link leaves
// through a wall, the equilibrium of the reversed direction at z itself.  Written by pushing:
// each cell evaluates its own 18 equilibria once and stores direction a at the cell it is pulled
// from, z - e_a, or, when that lies beyond a wall, as the reversed plane at itself (which the
// pull's bounce-back reads).  Every (plane, cell) is written exactly once.
template <int ST>
__global__ void k_init_pop(Phys P, Grid g, const float* __restrict__ fields) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  for (int y = blockIdx.y; y < g.ny; y += gridDim.y) {   // gridDim.y is capped at 65535
    const long long c = (long long)y * g.pitch + x;
    const float ph = fields[c], u = fields[2 * g.plane + c], v = fields[3 * g.plane + c];
    const float p = fields[4 * g.plane + c];
    // mu0 = theta'(phi0) - kappa lap(phi0) (Eq. 1); beyond a wall phi is mirrored (zero gradient)
    auto at = [&](int dx, int dy) {
      int xx = x + dx, yy = y + dy;
      xx = g.bc_x == BC_WALL ? mirror(xx, g.nx) : wrap1(xx, g.nx);
      yy = g.bc_y == BC_WALL ? mirror(yy, g.ny) : wrap1(yy, g.ny);
      return fields[(long long)yy * g.pitch + xx];
    };
    const float lap = (4.0f * (at(1, 0) + at(0, 1) + at(-1, 0) + at(0, -1)) +
                       (at(1, 1) + at(-1, 1) + at(-1, -1) + at(1, -1)) - 20.0f * ph) * (1.0f / 6.0f);
    const float m = P.four_beta * ph * (ph * ph - P.phi_star2) - P.kappa * lap;
    const float cl = fminf(fmaxf((ph + P.phi_star) * P.inv_2phistar, 0.0f), 1.0f);
    const float rho = P.rho_B + cl * P.drho;
    const float uu15 = 1.5f * (u * u + v * v);
    const CellB self = cell_at(y * g.row_bytes, col_bytes<ST>(x));
  #pragma unroll
    for (int a = 0; a < Q; ++a) {
      const float w = wgt(a);
      const float eu = (float)cx(a) * u + (float)cy(a) * v;
      const float poly = 3.0f * eu + 4.5f * eu * eu - uu15;
      const float geq = w * p + rho * (1.0f / 3.0f) * (w * poly);
      float feq = 0.0f;
      if (a > 0) feq = w * (P.f_forced ? ph * (1.0f + poly) : P.three_gamma_f * m + ph * poly);
      // where direction a's value is pulled from: z = this cell - e_a, or itself across a wall
      int xz = x - cx(a), yz = y - cy(a), plane = a;
      bool hit = false;
      if (xz < 0 || xz >= g.nx) {
        if (g.bc_x == BC_WALL) hit = true; else xz = wrap1(xz, g.nx);
      }
      if (yz < 0 || yz >= g.ny) {
        if (g.bc_y == BC_WALL) hit = true; else yz = wrap1(yz, g.ny);
      }
      if (hit) {
        xz = x;
        yz = y;
        plane = opp(a);
      }
      const CellB z = a == 0 ? self : cell_at(yz * g.row_bytes, col_bytes<ST>(xz));
      if (a == 0) {
        // f_0^eq = phi - sum_{k>0} f^eq_k, kept as the float pair (hi, lo)
        float rest = 0.0f;
  #pragma unroll
        for (int k = 1; k < Q; ++k) {
          const float ek = (float)cx(k) * u + (float)cy(k) * v;
          const float pk = 3.0f * ek + 4.5f * ek * ek - uu15;
          // f^eq_k: with the mu term, or phi Gamma_k in the forced order-parameter form
          rest += wgt(k) * (P.f_forced ? ph * (1.0f + pk) : P.three_gamma_f * m + ph * pk);
        }
        float hi, lo;
        two_sum(ph, -rest, hi, lo);
        if (ST == ST_FP32) {
          st_pop<ST>(g.dst, 0, self, hi, 1.0f);
          st_pop<ST>(g.dst, PLANE_F0LO, self, lo, 1.0f);
        } else {
          st_pop<ST>(g.dst, 0, self, hi + lo, 1.0f);
        }
      } else {
        st_pop<ST>(g.dst, plane, z, feq, g.sf);
      }
      st_pop<ST>(g.dst, Q + plane, z, geq, g.sg);
    }
  }
}

// s_form 1: rho and div(rho u) of the initial fields, which stand for the step before the first.
__global__ void k_init_sdef(Phys P, Grid g, const float* __restrict__ fields) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  for (int y = blockIdx.y; y < g.ny; y += gridDim.y) {   // gridDim.y is capped at 65535
    const float* phi = fields;
    const float* ux = fields + 2 * g.plane;
    const float* uy = fields + 3 * g.plane;
    auto idx = [&](int dx, int dy) {
      int xx = x + dx, yy = y + dy;
      xx = g.bc_x == BC_WALL ? mirror(xx, g.nx) : wrap1(xx, g.nx);
      yy = g.bc_y == BC_WALL ? mirror(yy, g.ny) : wrap1(yy, g.ny);
      return (long long)yy * g.pitch + xx;
    };
    auto rho = [&](long long i) { return fmad(__saturatef(fmad(phi[i], P.inv_2phistar, 0.5f)), P.drho, P.rho_B); };
    auto jx = [&](int dx, int dy) { const long long i = idx(dx, dy); return fmul(rho(i), ux[i]); };
    auto jy = [&](int dx, int dy) { const long long i = idx(dx, dy); return fmul(rho(i), uy[i]); };
    const float djx = fmad(4.0f, fsub(jx(1, 0), jx(-1, 0)), fsub(fsub(jx(1, 1), jx(-1, -1)), fsub(jx(-1, 1), jx(1, -1))));
    const float djy = fmad(4.0f, fsub(jy(0, 1), jy(0, -1)), fadd(fsub(jy(1, 1), jy(-1, -1)), fsub(jy(-1, 1), jy(1, -1))));
    float* sp = reinterpret_cast<float*>(static_cast<char*>(g.dst) + g.spoff);
    const long long c = (long long)y * g.pitch + x;
    sp[c] = rho(c);
    sp[g.plane + c] = fmul(fadd(djx, djy), 1.0f / 12.0f);
  }
}

cudaError_t launch_init(const lbm_sim* s, cudaStream_t st) {
  Grid g = make_grid(s, nullptr, s->buf[s->cur]);
  dim3 blk(128), grd((s->nx + 127) / 128, s->ny < 65535 ? s->ny : 65535);
  switch (g.storage) {
    case ST_FP16: k_init_pop<ST_FP16><<<grd, blk, 0, st>>>(s->phys, g, s->fields); break;
    case ST_BF16: k_init_pop<ST_BF16><<<grd, blk, 0, st>>>(s->phys, g, s->fields); break;
    default: k_init_pop<ST_FP32><<<grd, blk, 0, st>>>(s->phys, g, s->fields); break;
  }
  if (s->params.s_form) {
    cudaError_t e2 = cudaGetLastError();
    if (e2 != cudaSuccess) return e2;
    k_init_sdef<<<grd, blk, 0, st>>>(s->phys, g, s->fields);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 diagnostics
// Stage 1: one block per row, fixed per-thread stride and fixed tree -> 12 partials per row.
// Stage 2: one block folds the rows in a fixed order.  Results are bitwise reproducible.

constexpr int DIAG_T = 256;

__device__ __forceinline__ void tree_sum(double* sh, int t) {
  for (int s = DIAG_T / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
}
__device__ __forceinline__ void tree_max(double* sh, int t) {
  for (int s = DIAG_T / 2; s > 0; s >>= 1) {
    if (t < s) {
      const double a = sh[t], b = sh[t + s];
      sh[t] = (a >= b || a != a) ? a : b;   // NaN propagates
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(DIAG_T) k_diag_rows(Phys P, Grid g, const float* __restrict__ fields,
                                                      double* __restrict__ part) {
  __shared__ double sh[DIAG_PARTIALS][DIAG_T];
  const int y = blockIdx.x, t = threadIdx.x;
  const float* phi = fields + (long long)y * g.pitch;
  const float* ux = fields + 2 * g.plane + (long long)y * g.pitch;
  const float* uy = fields + 3 * g.plane + (long long)y * g.pitch;
  const float* pp = fields + 4 * g.plane + (long long)y * g.pitch;
  double acc[DIAG_PARTIALS] = {0};
  const double phs = P.phi_star;
  for (int x = t; x < g.nx; x += DIAG_T) {
    const double ph = phi[x], u = ux[x], v = uy[x], p = pp[x];
    double c = (ph + phs) / (2.0 * phs);
    c = c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
    acc[0] += ph;
    acc[1] += c;
    acc[2] += c * x;
    acc[3] += c * y;
    acc[4] += c * u;
    acc[5] += c * v;
    const double um = sqrt(u * u + v * v);
    if (!(um <= acc[6])) acc[6] = um;
    if (ph > 0.9 * phs) { acc[7] += p; acc[8] += 1.0; }
    if (ph < -0.9 * phs) { acc[9] += p; acc[10] += 1.0; }
  }
  for (int k = 0; k < 11; ++k) sh[k][t] = acc[k];
  __syncthreads();
  for (int k = 0; k < 11; ++k) {
    if (k == 6) tree_max(sh[k], t); else tree_sum(sh[k], t);
  }
  if (t < 11) part[(long long)y * DIAG_PARTIALS + t] = sh[t][0];
  if (t == 11) part[(long long)y * DIAG_PARTIALS + 11] = 0.0;
}

__global__ void __launch_bounds__(DIAG_T) k_diag_final(Grid g, const double* __restrict__ part,
                                                       double* __restrict__ out, long long step) {
  __shared__ double sh[DIAG_PARTIALS][DIAG_T];
  const int t = threadIdx.x;
  double acc[DIAG_PARTIALS] = {0};
  for (int y = t; y < g.ny; y += DIAG_T) {
    const double* r = part + (long long)y * DIAG_PARTIALS;
    for (int k = 0; k < 11; ++k) {
      if (k == 6) {
        if (!(r[6] <= acc[6])) acc[6] = r[6];
      } else {
        acc[k] += r[k];
      }
    }
    if (!(r[1] <= acc[11])) acc[11] = r[1];   // widest liquid chord
  }
  for (int k = 0; k < DIAG_PARTIALS; ++k) sh[k][t] = acc[k];
  __syncthreads();
  for (int k = 0; k < DIAG_PARTIALS; ++k) {
    if (k == 6 || k == 11) tree_max(sh[k], t); else tree_sum(sh[k], t);
  }
  if (t == 0) {
    lbm_diag d;
    d.step = step;
    d.sum_phi = sh[0][0];
    d.liquid_area = sh[1][0];
    const double sc = sh[1][0];
    d.centroid_x = sc > 0 ? sh[2][0] / sc : 0.0;
    d.centroid_y = sc > 0 ? sh[3][0] / sc : 0.0;
    d.vel_x = sc > 0 ? sh[4][0] / sc : 0.0;
    d.vel_y = sc > 0 ? sh[5][0] / sc : 0.0;
    d.spread_radius = 0.5 * sh[11][0];
    d.max_u = sh[6][0];
    d.p_liquid = sh[8][0] > 0 ? sh[7][0] / sh[8][0] : 0.0;
    d.p_gas = sh[10][0] > 0 ? sh[9][0] / sh[10][0] : 0.0;
    d.finite = isfinite(d.sum_phi) && isfinite(d.max_u);
    d.pad = 0;
    *reinterpret_cast<lbm_diag*>(out) = d;
  }
}

cudaError_t launch_diag(const lbm_sim* s, cudaStream_t st) {
  Grid g = make_grid(s, nullptr, nullptr);
  k_diag_rows<<<s->ny, DIAG_T, 0, st>>>(s->phys, g, s->fields, s->red);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_diag_final<<<1, DIAG_T, 0, st>>>(g, s->red, s->red + (long long)s->ny * DIAG_PARTIALS, s->steps);
  return cudaGetLastError();
}

}  // namespace lbm
