// Device side of the two-distribution D2Q9 multiphase lattice Boltzmann step for sm_103a.
//
// State layout in HBM (one simulation, one buffer of a ping-pong pair):
//   19 planes [f_0..f_8, gbar_0..gbar_8, f_0lo], each ny rows of `pitch` elements (pitch = nx
//   rounded up to 32 elements, so every row starts on a 128-byte boundary).  The planes hold
//   POST-collision populations at their source cell; a step pulls f_a(x) = f*_a(x - e_a) (or the
//   reversed population at a wall), computes the macroscopic fields, collides in registers and
//   writes f*_a(x) back at x: every global store is an aligned, coalesced row segment.
//   The rest population f_0 ~ phi is the only O(1) population; it is kept as an unevaluated
//   float pair f_0 + f_0lo (plane 18) so that phi, and through it mu and the surface-tension
//   force, carry ~2^-48 relative precision with FP32 arithmetic.  All other populations are
//   O(mu, u) and need no such care.
//
// The fused step kernel marches a CTA up a strip of columns.  One thread owns one column of the
// strip plus a 3-column halo on each side, and per row iteration runs four skewed stages whose
// results live in small shared-memory ring buffers of rows:
//   S0 row a    : phi = sum_a f_a                               (strip + 3 halo columns)
//   S1 row a-2  : mu = theta'(phi) - kappa lap(phi)               (strip + 2)     [Eq. 1]
//   S2 row a-4  : grad phi, grad mu, lap mu, rho, F_s, G, s, u, p (strip + 1)     [Eq. 4, 5, 8]
//   S3 row a-5  : grad p, grad psi, equilibria, forcing, BGK collisions of f and gbar, stores
// so every population is read from HBM once and every stencil works from shared memory.  The
// gathers of the next row (f for S0, gbar for S2) are issued one iteration ahead so their
// latency overlaps the current row's arithmetic; the populations S3 needs again wait in
// thread-private shared-memory rings.  One __syncthreads per row orders S2 -> S3; the ring
// sizes keep every other reader/writer pair on distinct rows.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int Q = 9;
constexpr int BC_PERIODIC = 0;
constexpr int BC_WALL = 1;

// D2Q9 ordering: rest, E, N, W, S, NE, NW, SW, SE.
__host__ __device__ constexpr int cx(int a) {
  return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int a) {
  return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int a) {
  return a == 0 ? 0 : (a <= 4 ? ((a + 1) & 3) + 1 : ((a - 3) & 3) + 5);
}
__host__ __device__ constexpr float wgt(int a) {
  return a == 0 ? 4.0f / 9.0f : (a <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "axis opposites");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "diagonal opposites");

// Scheme constants in FP32, derived once on the host from lbm_params.
struct Phys {
  float four_beta;      // 4 beta
  float kappa;
  float phi_star;
  float phi_star2;      // phi*^2
  float inv_2phistar;   // 1 / (2 phi*)
  float rho_B;
  float drho;           // rho_A - rho_B
  float rho_prime;      // (rho_A - rho_B) / (2 phi*)
  float s_coef;         // rho' theta_M
  float gravity;
  float omega_f;        // 1 / tau_f
  float three_gamma_f;  // 3 theta_M / (tau_f - 1/2)
  float mu_A, mu_B;     // dynamic viscosities rho_X cs2 (tau_g_X - 1/2)
  int remove_Fa;
};

// Geometry and buffers of one simulation as the kernels see them.
constexpr int N_PLANES = 19;   // f_0..f_8, gbar_0..gbar_8, f_0lo
constexpr int PLANE_F0LO = 18;

struct Grid {
  const float* src;     // post-collision state at t-1 (read)
  float* dst;           // post-collision state at t (write)
  int plane;            // elements per plane (ny * pitch); all planes fit in 2^31 elements
  int nx, ny, pitch;
  int bc_x, bc_y;
  int tile_w;           // interior columns per strip
  int seg_h;            // rows per segment
  int n_strips;
};

// Output planes of the moments mode (row-major with `pitch`).
struct MomentOut {
  float *phi, *rho, *ux, *uy, *p;
};

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}
// Mirror about a wall half a cell outside the edge: -1 -> 0, -2 -> 1, n -> n-1.
__device__ __forceinline__ int mirror(int i, int n) { return i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i); }

// Physical neighbourhood of one cell for the pull gather.
struct Cell {
  int xp, yp;            // the cell
  int xm, xq, ym, yq;    // columns x-1, x+1 and rows y-1, y+1 (wrapped)
  bool wl, wr, wb, wt;   // x-1 / x+1 / y-1 / y+1 lie beyond a wall
};

__device__ __forceinline__ Cell make_cell(int xp, int yp, const Grid& g) {
  Cell c;
  c.xp = xp;
  c.yp = yp;
  c.xm = xp == 0 ? g.nx - 1 : xp - 1;
  c.xq = xp == g.nx - 1 ? 0 : xp + 1;
  c.ym = yp == 0 ? g.ny - 1 : yp - 1;
  c.yq = yp == g.ny - 1 ? 0 : yp + 1;
  c.wl = g.bc_x == BC_WALL && xp == 0;
  c.wr = g.bc_x == BC_WALL && xp == g.nx - 1;
  c.wb = g.bc_y == BC_WALL && yp == 0;
  c.wt = g.bc_y == BC_WALL && yp == g.ny - 1;
  return c;
}

// Error-free sum of two floats: s + e == a + b exactly (round-to-nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Pull the 9 pre-collision populations of one distribution (planes base..base+8) at cell c:
// v[a] = P*_a(x - e_a), or P*_opp(a)(x) when x - e_a lies beyond a wall (half-way bounce-back).
__device__ __forceinline__ void gather9(const float* __restrict__ src, int plane, int pitch, const Cell& c,
                                        int base, float v[Q]) {
  const float* __restrict__ s0 = src + base * plane;
  const int rm = c.ym * pitch, r0 = c.yp * pitch, rq = c.yq * pitch;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int ex = cx(a), ey = cy(a);
    const bool hit = (ex == 1 && c.wl) || (ex == -1 && c.wr) || (ey == 1 && c.wb) || (ey == -1 && c.wt);
    const int sx = ex == 1 ? c.xm : (ex == -1 ? c.xq : c.xp);
    const int sr = ey == 1 ? rm : (ey == -1 ? rq : r0);
    const int i_pull = a * plane + sr + sx;
    const int i_back = opp(a) * plane + r0 + c.xp;
    v[a] = __ldg(s0 + (hit ? i_back : i_pull));
  }
}

// Per-cell record carried from S2 to S3 in registers.
struct Rec {
  float phi, mu, rho, ux, uy, Fx, Fy, drx, dry, omega_g;
};

constexpr int RING_PHI = 8;  // rows a-7..a
constexpr int RING = 4;      // mu, p
constexpr int RING_F = 6;    // f rows a-5..a awaiting S3 (thread-private)
constexpr int NF = Q + 1;    // f_0..f_8 and f_0lo

template <int NT>
struct Smem {
  float phi_hi[RING_PHI][NT];
  float phi_lo[RING_PHI][NT];
  float mu[RING][NT];
  float p[RING][NT];
  float f[RING_F][NF][NT];   // own column only: no barrier needed
  float g[2][Q][NT];         // own column only
};

enum { MODE_STEP = 0, MODE_MOMENTS = 1 };

// Collision of both distributions at one cell and store of the post-collision populations.
// f[] holds f_0..f_8 and f_0lo (index Q), gb[] gbar_0..gbar_8.
__device__ __forceinline__ void collide_store(const Phys& P, const Rec& r, float p, float gpx, float gpy,
                                              const float f[NF], const float gb[Q], float* __restrict__ dst,
                                              int plane, int cell) {
  const float dpsix = gpx - (1.0f / 3.0f) * r.drx;
  const float dpsiy = gpy - (1.0f / 3.0f) * r.dry;
  const float uu15 = 1.5f * (r.ux * r.ux + r.uy * r.uy);
  const float rho3 = r.rho * (1.0f / 3.0f);
  const float og = r.omega_g;
  const float src_g = 1.0f - 0.5f * og;
  const float of = P.omega_f;
  const float gmu = P.three_gamma_f * r.mu;
  float fsum = 0.0f, feqsum = 0.0f;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const float w = wgt(a);
    const float ex = (float)cx(a), ey = (float)cy(a);
    const float eu = ex * r.ux + ey * r.uy;
    const float poly = 3.0f * eu + 4.5f * eu * eu - uu15;     // omega_a(u)/w_a - 1
    const float gam = w + w * poly;                            // omega_a(u)
    const float gmw = w * poly;                                // omega_a(u) - w_a
    const float geq = w * p + rho3 * gmw;
    const float S = (ex - r.ux) * (r.Fx * gam - gmw * dpsix) + (ey - r.uy) * (r.Fy * gam - gmw * dpsiy);
    dst[(Q + a) * plane + cell] = gb[a] - og * (gb[a] - geq) + src_g * S;
    if (a > 0) {
      const float feq = w * (gmu + r.phi * poly);
      fsum += f[a];
      feqsum += feq;
      dst[a * plane + cell] = f[a] - of * (f[a] - feq);
    }
  }
  // f_0^eq - f_0 = (phi - f_0) - sum_{a>0} f^eq_a = sum_{a>0} (f_a - f^eq_a): small, exact inputs
  float hi, lo;
  two_sum(f[0], f[Q] + of * (fsum - feqsum), hi, lo);
  dst[cell] = hi;
  dst[PLANE_F0LO * plane + cell] = lo;
}

// The fused step (MODE_STEP) or the moment evaluation (MODE_MOMENTS) over one tile:
// columns [x0, x0 + tile_w) x rows [ya, yb) of one simulation.
template <int NT, int MODE>
__device__ __forceinline__ void run_tile(const Phys& P, const Grid& g, const MomentOut& mo, int strip, int seg,
                                         Smem<NT>& sm) {
  const int t = threadIdx.x;
  const int x0 = strip * g.tile_w;
  const int x_end = min(x0 + g.tile_w, g.nx);
  const int width = x_end - x0;
  const int ya = seg * g.seg_h;
  const int yb = min(ya + g.seg_h, g.ny);
  const int xl = x0 - 3 + t;                 // logical column (may lie outside [0, nx))
  const bool xwall = g.bc_x == BC_WALL;
  const bool ywall = g.bc_y == BC_WALL;
  const bool col_real = !xwall || (xl >= 0 && xl < g.nx);
  const int xp = wrap(xl, g.nx);
  const bool in_w3 = t < width + 6 && col_real;
  const bool in_w2 = t >= 1 && t < width + 5 && col_real;
  const bool in_w1 = t >= 2 && t < width + 4 && col_real;
  const bool in_w0 = t >= 3 && t < width + 3;
  // shared-memory column of the logical neighbour xl + d (ghost columns beyond a wall read
  // their mirror image)
  auto col = [&](int d) {
    int q = xl + d;
    if (xwall && (q < 0 || q >= g.nx)) q = mirror(q, g.nx);
    return q - (x0 - 3);
  };
  auto row = [&](int r) { return (ywall && (r < 0 || r >= g.ny)) ? mirror(r, g.ny) : r; };
  auto row_ok = [&](int r) { return !ywall || (r >= 0 && r < g.ny); };
  auto s0_active = [&](int r) { return r >= ya - 3 && r <= yb + 2 && in_w3 && row_ok(r); };
  auto s2_active = [&](int r) { return r >= ya - 1 && r <= yb && in_w1 && row_ok(r); };
  const int cm = col(-1), c0 = t, cp = col(1);

  // prefetched gathers: f (+ f_0lo) of the next S0 row, gbar of the next S2 row
  float fp[NF], gp[Q];
  auto fetch_f = [&](int r) {
    const Cell c = make_cell(xp, wrap(r, g.ny), g);
    gather9(g.src, g.plane, g.pitch, c, 0, fp);
    fp[Q] = __ldg(g.src + PLANE_F0LO * g.plane + c.yp * g.pitch + c.xp);
  };
  auto fetch_g = [&](int r) {
    const Cell c = make_cell(xp, wrap(r, g.ny), g);
    gather9(g.src, g.plane, g.pitch, c, Q, gp);
  };
  if (s0_active(ya - 3)) fetch_f(ya - 3);

  Rec cur{}, prev{};
  int fslot = 0;                             // (a - ya + 3) mod RING_F: ring slot of row a
  for (int a = ya - 3; a <= yb + 4; ++a) {
    // ---- S0: phi at row a (as an unevaluated pair hi + lo)
    if (s0_active(a)) {
      const float small = fp[Q] + (((fp[1] + fp[2]) + (fp[3] + fp[4])) + ((fp[5] + fp[6]) + (fp[7] + fp[8])));
      float hi, lo;
      two_sum(fp[0], small, hi, lo);
      sm.phi_hi[a & (RING_PHI - 1)][t] = hi;
      sm.phi_lo[a & (RING_PHI - 1)][t] = lo;
      if (MODE == MODE_STEP && in_w0 && a >= ya) {
#pragma unroll
        for (int k = 0; k < NF; ++k) sm.f[fslot][k][t] = fp[k];
      }
    }
    if (s0_active(a + 1)) fetch_f(a + 1);
    // ---- S1: mu at row a-2
    {
      const int r = a - 2;
      if (r >= ya - 2 && r <= yb + 1 && in_w2 && row_ok(r)) {
        const float* hs = sm.phi_hi[row(r - 1) & (RING_PHI - 1)];
        const float* h0 = sm.phi_hi[r & (RING_PHI - 1)];
        const float* hn = sm.phi_hi[row(r + 1) & (RING_PHI - 1)];
        const float* ls = sm.phi_lo[row(r - 1) & (RING_PHI - 1)];
        const float* l0 = sm.phi_lo[r & (RING_PHI - 1)];
        const float* ln = sm.phi_lo[row(r + 1) & (RING_PHI - 1)];
        const float H = h0[c0], L = l0[c0];
        // differences from the centre: exact for neighbouring values of like magnitude
        auto d = [&](const float* hr, const float* lr, int c) { return (hr[c] - H) + (lr[c] - L); };
        const float lap = (4.0f * ((d(h0, l0, cp) + d(hn, ln, c0)) + (d(h0, l0, cm) + d(hs, ls, c0))) +
                           ((d(hn, ln, cp) + d(hn, ln, cm)) + (d(hs, ls, cm) + d(hs, ls, cp)))) * (1.0f / 6.0f);
        const float ph = H + L;
        const float dm = (H - P.phi_star) + L, dp = (H + P.phi_star) + L;
        sm.mu[r & (RING - 1)][t] = P.four_beta * ph * dm * dp - P.kappa * lap;
      }
    }
    // ---- S2: u, p at row a-4
    {
      const int r = a - 4;
      if (s2_active(r)) {
        const int rs_ = row(r - 1) & (RING_PHI - 1), r0_ = r & (RING_PHI - 1), rn_ = row(r + 1) & (RING_PHI - 1);
        const float* hs = sm.phi_hi[rs_];
        const float* h0 = sm.phi_hi[r0_];
        const float* hn = sm.phi_hi[rn_];
        const float* ls = sm.phi_lo[rs_];
        const float* l0 = sm.phi_lo[r0_];
        const float* ln = sm.phi_lo[rn_];
        const float* ms = sm.mu[row(r - 1) & (RING - 1)];
        const float* m0 = sm.mu[r & (RING - 1)];
        const float* mn = sm.mu[row(r + 1) & (RING - 1)];
        auto D = [&](const float* ha, const float* la, int ca, const float* hb, const float* lb, int cb) {
          return (ha[ca] - hb[cb]) + (la[ca] - lb[cb]);
        };
        const float ph = h0[c0] + l0[c0];
        const float gphx = (4.0f * D(h0, l0, cp, h0, l0, cm) + (D(hn, ln, cp, hn, ln, cm) + D(hs, ls, cp, hs, ls, cm))) *
                           (1.0f / 12.0f);
        const float gphy = (4.0f * D(hn, ln, c0, hs, ls, c0) + (D(hn, ln, cp, hs, ls, cp) + D(hn, ln, cm, hs, ls, cm))) *
                           (1.0f / 12.0f);
        const float gmx = (4.0f * (m0[cp] - m0[cm]) + (mn[cp] - mn[cm] - ms[cm] + ms[cp])) * (1.0f / 12.0f);
        const float gmy = (4.0f * (mn[c0] - ms[c0]) + (mn[cp] + mn[cm] - ms[cm] - ms[cp])) * (1.0f / 12.0f);
        const float cl = fminf(fmaxf((ph + P.phi_star) * P.inv_2phistar, 0.0f), 1.0f);
        const float rho = P.rho_B + cl * P.drho;
        const float fsx = -ph * gmx;
        const float fsy = -ph * gmy;
        const float gy = -rho * P.gravity;
        float sdef = 0.0f;
        if (P.remove_Fa) {
          const float lmu = (4.0f * (m0[cp] + mn[c0] + m0[cm] + ms[c0]) + (mn[cp] + mn[cm] + ms[cm] + ms[cp]) -
                             20.0f * m0[c0]) * (1.0f / 6.0f);
          sdef = P.s_coef * lmu;
        }
        const float* gb = gp;
        const float m0g = ((gb[0] + gb[1]) + (gb[2] + gb[3])) + ((gb[4] + gb[5]) + (gb[6] + gb[7])) + gb[8];
        const float jx = (gb[1] - gb[3]) + (gb[5] - gb[6]) + (gb[8] - gb[7]);
        const float jy = (gb[2] - gb[4]) + (gb[5] + gb[6]) - (gb[7] + gb[8]);
        const float denom = P.remove_Fa ? rho - 0.5f * sdef : rho;
        const float ux = (3.0f * jx + 0.5f * fsx) / denom;
        const float uy = (3.0f * jy + 0.5f * (fsy + gy)) / denom;
        const float drx = P.rho_prime * gphx, dry = P.rho_prime * gphy;
        const float p = m0g + (1.0f / 6.0f) * (ux * drx + uy * dry);
        sm.p[r & (RING - 1)][t] = p;
        if (MODE == MODE_MOMENTS) {
          if (in_w0 && r >= ya && r < yb) {
            const int o = r * g.pitch + xp;
            mo.phi[o] = ph;
            mo.rho[o] = rho;
            mo.ux[o] = ux;
            mo.uy[o] = uy;
            mo.p[o] = p;
          }
        } else {
          if (in_w0 && r >= ya) {
#pragma unroll
            for (int k = 0; k < Q; ++k) sm.g[r & 1][k][t] = gb[k];
          }
          cur.phi = ph;
          cur.mu = m0[c0];
          cur.rho = rho;
          cur.ux = ux;
          cur.uy = uy;
          cur.Fx = fsx + (P.remove_Fa ? ux * sdef : 0.0f);
          cur.Fy = fsy + gy + (P.remove_Fa ? uy * sdef : 0.0f);
          cur.drx = drx;
          cur.dry = dry;
          const float muv = P.mu_B + cl * (P.mu_A - P.mu_B);
          cur.omega_g = 1.0f / (3.0f * muv / rho + 0.5f);
        }
      }
      if (s2_active(r + 1)) fetch_g(r + 1);
    }
    __syncthreads();
    // ---- S3: collide and store row a-5
    if (MODE == MODE_STEP) {
      const int r = a - 5;
      if (r >= ya && r < yb && in_w0) {
        const float* qs = sm.p[row(r - 1) & (RING - 1)];
        const float* q0 = sm.p[r & (RING - 1)];
        const float* qn = sm.p[row(r + 1) & (RING - 1)];
        const float gpx = (4.0f * (q0[cp] - q0[cm]) + (qn[cp] - qn[cm] - qs[cm] + qs[cp])) * (1.0f / 12.0f);
        const float gpy = (4.0f * (qn[c0] - qs[c0]) + (qn[cp] + qn[cm] - qs[cm] - qs[cp])) * (1.0f / 12.0f);
        const int rslot = fslot == RING_F - 1 ? 0 : fslot + 1;   // row a-5 == row a+1 (mod 6)
        float f[NF], gb[Q];
#pragma unroll
        for (int k = 0; k < NF; ++k) f[k] = sm.f[rslot][k][t];
#pragma unroll
        for (int k = 0; k < Q; ++k) gb[k] = sm.g[r & 1][k][t];
        collide_store(P, prev, q0[c0], gpx, gpy, f, gb, g.dst, g.plane, r * g.pitch + xp);
      }
    }
    prev = cur;
    fslot = fslot == RING_F - 1 ? 0 : fslot + 1;
  }
}

}  // namespace lbm
