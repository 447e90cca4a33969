// Device side of the two-distribution D2Q9 multiphase lattice Boltzmann step for sm_103a.
//
// State layout in HBM (one simulation, one buffer of a ping-pong pair):
//   19 population planes [f_0..f_8, gbar_0..gbar_8, f_0lo], stored in blocks of 32 cells: a row
//   of the grid is pitch / 32 consecutive blocks (pitch = nx rounded up to 32), and a block holds
//   the 32 cells' values of every plane, plane after plane (FP32: 19 x 128 B = 2432 B).  The
//   offset of a plane inside a block is a compile-time constant, so one byte offset per (row,
//   column) addresses all populations of a cell, and a warp's access to one plane of 32
//   consecutive cells is one or two aligned 128-byte segments.  The planes hold POST-collision
//   populations at their source cell; a step pulls f_a(x) = f*_a(x - e_a) (or the reversed
//   population at a wall), computes the macroscopic fields, collides in registers and writes
//   f*_a(x) back at x: every global store is an aligned, coalesced segment.
//   The rest population f_0 ~ phi is the only O(1) population; it is kept as an unevaluated
//   float pair f_0 + f_0lo (plane 18) so that phi, and through it mu and the surface-tension
//   force, carry ~2^-48 relative precision with FP32 arithmetic.  All other populations are
//   O(mu, u) and need no such care.
//   With the direct mass defect (s_form 1) each buffer also holds, after the populations, two
//   FP32 planes [rho, div(rho u)] of the step that wrote it, each ny rows of `pitch` elements.
//
// The fused step kernel marches a CTA up a strip of columns.  One thread owns one column of the
// strip plus a 3-column halo on each side, and per row iteration runs four skewed stages whose
// results live in small shared-memory ring buffers of rows:
//   S0 row a    : phi = sum_a f_a                               (strip + 3 halo columns)
//   S1 row a-2  : mu = theta'(phi) - kappa lap(phi)               (strip + 2)     [Eq. 1]
//   S2 row a-4  : grad phi, grad mu, lap mu, rho, F_s, G, s, u, p (strip + 1)     [Eq. 4, 5, 8]
//   S3 row a-5  : grad p, grad psi, div u (convective Cahn-Hilliard source), equilibria,
//                 forcing, BGK collisions of f and gbar, stores
// so every population is read from HBM once and every stencil works from shared memory.  The
// gathers of the next row (f for S0, gbar for S2) are issued one iteration ahead so their
// latency overlaps the current row's arithmetic; the populations S3 needs again wait in
// thread-private shared-memory rings.  One __syncthreads per row orders S2 -> S3; the ring
// sizes keep every other reader/writer pair on distinct rows.  The pipeline fill and drain and
// the iterations that touch a boundary row run a checked body; interior iterations run one with
// no row tests.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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
  // folded into the step kernel's arithmetic
  float kappa6;         // kappa / 6 (the isotropic Laplacian carries 1/6)
  float rho_prime12;    // rho' / 12 (the isotropic gradient carries 1/12)
  float s_coef6;        // rho' theta_M / 6
  float mu3_B, mu3_d;   // 3 mu_B and 3 (mu_A - mu_B)
  float keep_f;         // 1 - omega_f
  float of3gf;          // omega_f 3 Gamma_f
  int ch_conv;          // 1: the f collision adds w_a phi div(u) (convective Cahn-Hilliard form)
  int fs_mu;            // 1: F_s = mu grad(phi); 0: F_s = -phi grad(mu)
  int s_direct;         // 1: s = (rho - rho_prev) + div(rho u)_prev from the state's extra planes
  int f_forced;         // 1: forced order-parameter LBE (equilibrium phi Gamma_a)
  float hf12;           // (1 - omega_f / 2) / 12: weight of its grad(phi) forcing (12 grad phi)
  float thM6;           // theta_M / 6: its mobility source from 6 lap(mu)
};

// Geometry and buffers of one simulation as the kernels see them.
constexpr int N_PLANES = 19;   // FP32 storage: f_0..f_8, gbar_0..gbar_8, f_0lo
constexpr int PLANE_F0LO = 18;

// Population storage.  FP32: 19 float planes (f_0 as the pair f_0 + f_0lo).  FP16 / BF16: the
// rest population f_0 ~ phi stays one float plane (16-bit rounding of an O(1) value would
// drift phi by ~1e-4 per step); the 17 other populations, all O(mu, u), are 16-bit planes
// after it, stored as value x scale (a power of two keeping FP16 in its normal range).
constexpr int ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2;

__host__ __device__ constexpr long long state_bytes_per_cell(int st) { return st == ST_FP32 ? 4 * N_PLANES : 4 + 2 * 17; }

// Blocked layout: 32 cells per block.  FP32: 19 planes of 128 B.  16-bit: the FP32 rest plane
// (128 B), then 17 planes of 64 B.
constexpr int BLK = 32;
__host__ __device__ constexpr int block_bytes(int st) { return (int)state_bytes_per_cell(st) * BLK; }
// Byte offset of plane a inside a block (lane 0).
template <int ST>
__host__ __device__ constexpr int plane_off(int a) {
  return ST == ST_FP32 ? a * BLK * 4 : (a == 0 ? 0 : BLK * 4 + (a - 1) * BLK * 2);
}
// Byte offsets of one cell's lane inside the population region: `b4` for 4-byte planes (every
// plane in FP32; the rest plane in 16-bit storage), `b2` for the 2-byte planes.
struct CellB {
  int b4, b2;
};

struct Grid {
  const void* src;      // post-collision state at t-1 (read)
  void* dst;            // post-collision state at t (write)
  int plane;            // elements per plane of the s_form planes (ny * pitch)
  int row_bytes;        // bytes per population row: pitch / 32 blocks (the region fits in 2^31 bytes)
  int storage;          // ST_FP32 / ST_FP16 / ST_BF16
  float sf, isf;        // 16-bit scale of the f planes and its inverse
  float sg, isg;        // 16-bit scale of the gbar planes and its inverse
  int nx, ny, pitch;
  int bc_x, bc_y;
  int tile_w;           // interior columns per strip
  int seg_h;            // rows per segment
  int n_strips;
  long long spoff;      // s_form 1: byte offset of the [rho, div(rho u)] planes in src/dst (else 0)
};

// Output planes of the moment pass (row-major with `pitch`); each may be null.  fax, fay: the
// additional interfacial force F_a = -u s of Eq. 12 (s by the simulation's s_form), evaluated
// whichever scheme runs.
struct MomentOut {
  float *phi, *rho, *ux, *uy, *p;
  float *fax, *fay;
};

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}
// Mirror about a wall half a cell outside the edge: -1 -> 0, -2 -> 1, n -> n-1.
__device__ __forceinline__ int mirror(int i, int n) { return i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i); }

// Wrap an index that lies within one period of [0, n) (the general case takes a modulo).
__device__ __forceinline__ int wrap1(int i, int n) {
  if (i < -n || i >= 2 * n) return wrap(i, n);
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Byte offsets of column x inside a population row.
template <int ST>
__host__ __device__ __forceinline__ CellB col_bytes(int x) {
  const int blk = (x >> 5) * block_bytes(ST), lane = x & (BLK - 1);
  return CellB{blk + lane * 4, blk + lane * 2};
}
__host__ __device__ __forceinline__ CellB cell_at(int row_off, CellB c) { return CellB{row_off + c.b4, row_off + c.b2}; }

// Column part of one thread's pull neighbourhood (fixed for the whole tile).
struct ColNb {
  int xm, x0, xq;      // physical columns of x-1, x, x+1 (wrapped)
  CellB cm, c0, cq;    // their byte offsets inside a population row
  bool wl, wr;         // x-1 / x+1 lie beyond a wall
};
// Row part of the neighbourhood of one gathered row.
struct RowNb {
  int rm, r0, rq;      // element offsets (row * pitch) of rows y-1, y, y+1 (wrapped): s_form planes
  int bm, b0, bq;      // byte offsets (row * row_bytes) of the same rows in the population region
  bool wb, wt;         // y-1 / y+1 lie beyond a wall
};

template <int ST>
__device__ __forceinline__ ColNb make_col(int xp, const Grid& g) {
  ColNb c;
  c.x0 = xp;
  c.xm = xp == 0 ? g.nx - 1 : xp - 1;
  c.xq = xp == g.nx - 1 ? 0 : xp + 1;
  c.cm = col_bytes<ST>(c.xm);
  c.c0 = col_bytes<ST>(c.x0);
  c.cq = col_bytes<ST>(c.xq);
  c.wl = g.bc_x == BC_WALL && xp == 0;
  c.wr = g.bc_x == BC_WALL && xp == g.nx - 1;
  return c;
}

__device__ __forceinline__ RowNb make_row(int yp, const Grid& g) {
  RowNb r;
  r.r0 = yp * g.pitch;
  r.rm = yp == 0 ? (g.ny - 1) * g.pitch : r.r0 - g.pitch;
  r.rq = yp == g.ny - 1 ? 0 : r.r0 + g.pitch;
  r.b0 = yp * g.row_bytes;
  r.bm = yp == 0 ? (g.ny - 1) * g.row_bytes : r.b0 - g.row_bytes;
  r.bq = yp == g.ny - 1 ? 0 : r.b0 + g.row_bytes;
  r.wb = g.bc_y == BC_WALL && yp == 0;
  r.wt = g.bc_y == BC_WALL && yp == g.ny - 1;
  return r;
}

// Error-free sum of two floats: s + e == a + b exactly (round-to-nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Population a (0..8 f, 9..17 gbar, 18 f_0lo) of the cell at byte offsets c, as stored bits (a
// float, or a 16-bit value in the low half), and their decoding.  A prefetch keeps the bits and
// decodes them where they are used, so that the conversion does not wait for the load at the
// point of issue.  COH: a kernel that reads state other CTAs write during the same launch loads
// through L2 only (ld.global.cg, ordered by the memory model); every other kernel takes the
// read-only path.
template <int ST, bool COH = false>
__device__ __forceinline__ unsigned int ld_raw(const void* __restrict__ base, int a, CellB c) {
  const char* p = static_cast<const char*>(base) + plane_off<ST>(a);
  if (ST == ST_FP32 || a == 0) {
    const float* q = reinterpret_cast<const float*>(p + c.b4);
    return __float_as_uint(COH ? __ldcg(q) : __ldg(q));
  }
  const unsigned short* q = reinterpret_cast<const unsigned short*>(p + c.b2);
  return COH ? __ldcg(q) : __ldg(q);
}

// Decoded populations stay in their storage scale: a 16-bit plane (a > 0) holds the population
// times a power of two (4096 for FP16, 1 for BF16), and the step carries that scale through its
// linear arithmetic instead of multiplying every value: the sums of S0 and S2 are unscaled once
// per cell, the collision's per-cell constants are scaled once.  Scaling by a power of two is
// exact, so every result is bitwise the one of unscaled arithmetic.
template <int ST>
__device__ __forceinline__ float dec_pop(unsigned int raw, int a) {
  if (ST == ST_FP32 || a == 0) return __uint_as_float(raw);
  const unsigned short r16 = static_cast<unsigned short>(raw);
  return ST == ST_FP16 ? __half2float(__ushort_as_half(r16)) : __bfloat162float(__ushort_as_bfloat16(r16));
}

// BF16 bits of v by stochastic rounding: a pseudo-random 16-bit offset is added to the 16 bits
// that truncation drops, so v rounds away from zero with probability equal to the dropped
// fraction and the rounding error has zero mean.  Round-to-nearest at BF16's 8-bit significand
// biases the gbar populations, which change little from step to step, the same way every step:
// a falling drop's centroid velocity drifted by 3.6 %.  Unbiased rounding of the gbar planes
// keeps it within 0.05 %; the f planes round to nearest (rounding them stochastically as well
// gained nothing, and rounding only them left the 3.6 %).
// The offset is a hash of the value's own bits and its storage address, so every kernel rounds a
// given value at a given place alike and runs stay deterministic.  NaN and infinity keep round-to-nearest, so a diverged state stays
// non-finite.
__device__ __forceinline__ unsigned short bf16_stochastic(float v, unsigned int where) {
  const unsigned int bits = __float_as_uint(v);
  if ((bits & 0x7f800000u) == 0x7f800000u) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  // the high half of a product with an odd constant depends on every bit of the other factor
  const unsigned int offset = ((bits ^ where) * 0x9e3779b1u) >> 16;
  return static_cast<unsigned short>((bits + offset) >> 16);
}

// Store population a given in storage scale (16-bit planes) or as is (FP32, the rest plane).
template <int ST>
__device__ __forceinline__ void st_pop_scaled(void* __restrict__ base, int a, CellB c, float sv) {
  char* p = static_cast<char*>(base) + plane_off<ST>(a);
  if (ST == ST_FP32 || a == 0) {
    *reinterpret_cast<float*>(p + c.b4) = sv;
  } else if (ST == ST_FP16) {
    *reinterpret_cast<unsigned short*>(p + c.b2) = __half_as_ushort(__float2half_rn(sv));
  } else if (a >= Q) {   // gbar: stochastic rounding (see bf16_stochastic)
    *reinterpret_cast<unsigned short*>(p + c.b2) =
        bf16_stochastic(sv, static_cast<unsigned int>(c.b2 + plane_off<ST>(a)));
  } else {                // f: round to nearest meets the bound
    *reinterpret_cast<unsigned short*>(p + c.b2) = __bfloat16_as_ushort(__float2bfloat16_rn(sv));
  }
}

// Store population a given unscaled (the initial state).
template <int ST>
__device__ __forceinline__ void st_pop(void* __restrict__ base, int a, CellB c, float v, float scale) {
  st_pop_scaled<ST>(base, a, c, (ST == ST_FP32 || a == 0) ? v : __fmul_rn(v, scale));
}

// Multiply by a storage scale only where populations are stored in 16 bits.
template <int ST>
__device__ __forceinline__ float to_scale(float v, float scale) {
  return ST == ST_FP32 ? v : __fmul_rn(v, scale);
}

// Pull the 9 pre-collision populations of one distribution (planes starting at `src`), as stored
// bits (decode with dec_pop at plane FIRST + a):
// v[a] = P*_a(x - e_a), or P*_opp(a)(x) when x - e_a lies beyond a wall (half-way bounce-back).
// Cells with no wall neighbour take the branch-free path.
template <int ST, int FIRST, bool COH = false>
__device__ __forceinline__ void gather9(const void* __restrict__ src, const ColNb& c, const RowNb& r, unsigned int v[Q]) {
  if (!(c.wl | c.wr | r.wb | r.wt)) {
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const CellB sx = cx(a) == 1 ? c.cm : (cx(a) == -1 ? c.cq : c.c0);
      const int sr = cy(a) == 1 ? r.bm : (cy(a) == -1 ? r.bq : r.b0);
      v[a] = ld_raw<ST, COH>(src, FIRST + a, cell_at(sr, sx));
    }
  } else {
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const int ex = cx(a), ey = cy(a);
      const bool hit = (ex == 1 && c.wl) || (ex == -1 && c.wr) || (ey == 1 && r.wb) || (ey == -1 && r.wt);
      const CellB sx = ex == 1 ? c.cm : (ex == -1 ? c.cq : c.c0);
      const int sr = ey == 1 ? r.bm : (ey == -1 ? r.bq : r.b0);
      v[a] = hit ? ld_raw<ST, COH>(src, FIRST + opp(a), cell_at(r.b0, c.c0)) : ld_raw<ST, COH>(src, FIRST + a, cell_at(sr, sx));
    }
  }
}

// Every floating-point operation of the step is an explicit round-to-nearest intrinsic, so no
// multiply-add contraction is left to the compiler: the inlined tile body computes bit for bit
// the same in the single-simulation kernel and in the batch kernel.
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// e_a . v from the precomputed projections vx, vy, vx + vy, vx - vy (no arithmetic).
template <int A>
__device__ __forceinline__ float eproj(float vx, float vy, float vp, float vm) {
  return A == 1 ? vx : A == 2 ? vy : A == 3 ? -vx : A == 4 ? -vy : A == 5 ? vp : A == 6 ? -vm : A == 7 ? -vp : vm;
}

// Isotropic gradient of a 3x3 stencil, times 12: rows s (south), 0, n (north), columns -1, 0, +1.
//   12 dq/dx = 4 (E - W) + (NE - NW) + (SE - SW) = 4 (E - W) + (d1 - d2)
//   12 dq/dy = 4 (N - S) + (NE - SE) + (NW - SW) = 4 (N - S) + (d1 + d2),  d1 = NE - SW, d2 = NW - SE
__device__ __forceinline__ void grad12(const float* s, const float* c, const float* n, float& gx, float& gy) {
  const float d1 = fsub(n[1], s[-1]), d2 = fsub(n[-1], s[1]);
  gx = fmad(4.0f, fsub(c[1], c[-1]), fsub(d1, d2));
  gy = fmad(4.0f, fsub(n[0], s[0]), fadd(d1, d2));
}

// Per-cell record carried from S2 to S3 in registers.
struct Rec {
  float phi, mu, ux, uy, Fx, Fy;
  float mrx3, mry3;     // -(grad rho) / 3
  float og;             // omega_g = 1 / tau_g(phi)
  float ogr3;           // omega_g rho / 3
  float gx12, gy12;     // forced order-parameter form: 12 grad(phi)
  float lmu6;           // and 6 lap(mu)
};

constexpr int RING = 8;      // rows of phi (hi, lo), mu and p, incl. one mirrored ghost row at a wall
constexpr int RING_U = 4;    // rows of u_x, u_y (written by S2 at a-4, read by S3 at a-6 .. a-4),
                             // plus two slots for the mirrored ghost rows beyond walls
constexpr int RING_F = 6;    // f rows a-5..a awaiting S3 (thread-private)
constexpr int NF = Q + 1;    // gathered f_0..f_8 and f_0lo
constexpr int NFR = 8;       // f_1..f_8 kept for S3: f_0 is rebuilt there from the phi pair

// Row ring fields, interleaved per slot so that one slot offset serves every field.
enum { R_PHI_HI = 0, R_PHI_LO = 1, R_MU = 2, R_P = 3, R_FIELDS = 4 };

template <int NT>
struct Smem {
  float rows[RING][R_FIELDS][NT];  // phi (hi, lo), mu, p of recent rows
  float urows[RING_U + 2][2][NT];  // u_x, u_y of recent rows (convective form only)
  float2 f[RING_F][NT][NFR / 2];   // own column only (no barrier needed); 64-bit accesses
  float g[2][Q][NT];               // own column only; the S2 -> S3 gbar of kernels without GREG
};

enum { MODE_STEP = 0, MODE_MOMENTS = 1 };

// Both collisions at one cell.  With Gamma_a = omega_a(u) = w_a (1 + poly_a),
// poly_a = 3 e.u + 4.5 (e.u)^2 - 1.5 u.u, gmw_a = Gamma_a - w_a = w_a poly_a, D = F - grad psi:
//   g^eq_a = w_a p + (rho / 3) gmw_a
//   S_a    = (e_a - u).[F Gamma_a - gmw_a grad psi] = w_a (e_a.F - u.F) + gmw_a (e_a.D - u.D)
//   gbar*_a = (1 - omega_g) gbar_a + omega_g g^eq_a + (1 - omega_g / 2) S_a
//   f*_a   = (1 - omega_f) f_a + omega_f w_a (3 Gamma_f mu + phi poly_a) + w_a phi div(u)   (a > 0)
// or, in the forced order-parameter form (FF), with h = 1 - omega_f / 2:
//   f*_a   = (1 - omega_f) f_a + Gamma_a [omega_f phi + h (e_a - u).grad phi + theta_M lap mu]
//            + w_a phi div(u)
// The weight-class products are formed once per cell (class 0: rest, 1: axis, 2: diagonal).
struct CollideC {
  float ux, uy, up, um, m15uu;
  float Fx, Fy, Fp, Fm;
  float Dx, Dy, Dp, Dm, uD;
  float wuF[3];     // -w_c u.F
  float A[3];       // omega_g w_c p
  float ogr3, keep_g, src_g, keep_f;
  float ofwg[3];    // omega_f w_c 3 Gamma_f mu
  float ofwp[3];    // omega_f w_c phi
  float hgx, hgy, hgp, hgm, c0, ofp;   // FF: h grad(phi) projections; theta_M lap mu - h u.grad phi; omega_f phi
  float wphiD[3];   // FF: w_c phi div(u)
};

// PART: COLLIDE_BOTH, or only the gbar (COLLIDE_G) or only the f (COLLIDE_F) populations, each
// computed exactly as in the joint form (the small-grid kernel gives them to two threads).
constexpr int COLLIDE_BOTH = 0, COLLIDE_F = 1, COLLIDE_G = 2;

template <int ST, int A, bool FF, int PART = COLLIDE_BOTH>
__device__ __forceinline__ void collide_dir(const CollideC& k, const float f[Q], const float gb[Q], const Grid& g,
                                            CellB cell, float& fsum, float& ofeqsum) {
  constexpr int C = A == 0 ? 0 : (A <= 4 ? 1 : 2);
  constexpr float w = wgt(A);
  float poly, t1w, t2;
  if (A == 0) {
    poly = k.m15uu;
    t1w = k.wuF[0];
    t2 = -k.uD;
  } else {
    const float eu = eproj<A>(k.ux, k.uy, k.up, k.um);
    poly = fmad(eu, fmad(4.5f, eu, 3.0f), k.m15uu);
    t1w = fmad(w, eproj<A>(k.Fx, k.Fy, k.Fp, k.Fm), k.wuF[C]);
    t2 = fsub(eproj<A>(k.Dx, k.Dy, k.Dp, k.Dm), k.uD);
  }
  const float gmw = fmul(w, poly);
  if (PART != COLLIDE_F) {
    const float S = fmad(gmw, t2, t1w);
    st_pop_scaled<ST>(g.dst, Q + A, cell, fmad(k.src_g, S, fmad(k.ogr3, gmw, fmad(k.keep_g, gb[A], k.A[C]))));
  }
  if (A > 0 && PART != COLLIDE_G) {
    float ofeq;
    if constexpr (FF) {
      const float Ga = fadd(w, gmw);                                        // Gamma_a
      const float ta = fadd(eproj<A>(k.hgx, k.hgy, k.hgp, k.hgm), k.c0);    // h (e_a - u).grad phi + theta_M lap mu
      ofeq = fmad(Ga, fadd(ta, k.ofp), k.wphiD[C]);
    } else {
      ofeq = fmad(k.ofwp[C], poly, k.ofwg[C]);
    }
    fsum = fadd(fsum, f[A]);
    ofeqsum = fadd(ofeqsum, ofeq);
    st_pop_scaled<ST>(g.dst, A, cell, fmad(k.keep_f, f[A], ofeq));
  }
}

// Collision of both distributions at one cell and store of the post-collision populations.
// f[] holds f_1..f_8 (index 0 unused), gb[] gbar_0..gbar_8; gpx12/gpy12 are 12 grad p.
// phiD = phi div(u) (convective form) or 0: the f collision adds w_a phiD to direction a.
template <int ST, bool FF, int PART = COLLIDE_BOTH>
__device__ __forceinline__ void collide_store(const Phys& P, const Rec& r, float p, float gpx12, float gpy12,
                                              float phi_hi, float phi_lo, float phiD, const float f[Q],
                                              const float gb[Q], const Grid& g, CellB cell) {
  CollideC k;
  k.ux = r.ux;
  k.uy = r.uy;
  k.up = fadd(r.ux, r.uy);
  k.um = fsub(r.ux, r.uy);
  k.m15uu = fmul(-1.5f, fmad(r.ux, r.ux, fmul(r.uy, r.uy)));
  k.Fx = r.Fx;
  k.Fy = r.Fy;
  k.Fp = fadd(r.Fx, r.Fy);
  k.Fm = fsub(r.Fx, r.Fy);
  // grad psi = grad p - cs2 grad rho
  k.Dx = fsub(r.Fx, fmad(gpx12, 1.0f / 12.0f, r.mrx3));
  k.Dy = fsub(r.Fy, fmad(gpy12, 1.0f / 12.0f, r.mry3));
  k.Dp = fadd(k.Dx, k.Dy);
  k.Dm = fsub(k.Dx, k.Dy);
  k.uD = fmad(r.ux, k.Dx, fmul(r.uy, k.Dy));
  const float uF = fmad(r.ux, r.Fx, fmul(r.uy, r.Fy));
  k.wuF[0] = fmul(-4.0f / 9.0f, uF);
  k.wuF[1] = fmul(-1.0f / 9.0f, uF);
  k.wuF[2] = fmul(-1.0f / 36.0f, uF);
  // terms added to a stored (16-bit: scaled) population carry the storage scale
  const float ogp = fmul(r.og, p);
  k.A[0] = to_scale<ST>(fmul(4.0f / 9.0f, ogp), g.sg);
  k.A[1] = to_scale<ST>(fmul(1.0f / 9.0f, ogp), g.sg);
  k.A[2] = to_scale<ST>(fmul(1.0f / 36.0f, ogp), g.sg);
  k.ogr3 = to_scale<ST>(r.ogr3, g.sg);
  k.keep_g = fsub(1.0f, r.og);
  k.src_g = to_scale<ST>(fmad(-0.5f, r.og, 1.0f), g.sg);
  k.keep_f = P.keep_f;
  const float ofg = fadd(fmul(P.of3gf, r.mu), phiD), ofp = fmul(P.omega_f, r.phi);
  k.ofwg[0] = k.ofwp[0] = 0.0f;
  k.ofwg[1] = to_scale<ST>(fmul(1.0f / 9.0f, ofg), g.sf);
  k.ofwg[2] = to_scale<ST>(fmul(1.0f / 36.0f, ofg), g.sf);
  k.ofwp[1] = to_scale<ST>(fmul(1.0f / 9.0f, ofp), g.sf);
  k.ofwp[2] = to_scale<ST>(fmul(1.0f / 36.0f, ofp), g.sf);
  if constexpr (FF) {
    const float hx = fmul(P.hf12, r.gx12), hy = fmul(P.hf12, r.gy12);
    k.hgx = hx;
    k.hgy = hy;
    k.hgp = fadd(hx, hy);
    k.hgm = fsub(hx, hy);
    k.c0 = fsub(fmul(P.thM6, r.lmu6), fmad(r.ux, hx, fmul(r.uy, hy)));
    k.ofp = ofp;
    k.wphiD[0] = 0.0f;
    k.wphiD[1] = fmul(1.0f / 9.0f, phiD);
    k.wphiD[2] = fmul(1.0f / 36.0f, phiD);
  }
  float fsum = 0.0f, ofeqsum = 0.0f;
  collide_dir<ST, 0, FF, PART>(k, f, gb, g, cell, fsum, ofeqsum);
  collide_dir<ST, 1, FF, PART>(k, f, gb, g, cell, fsum, ofeqsum);
  collide_dir<ST, 2, FF, PART>(k, f, gb, g, cell, fsum, ofeqsum);
  collide_dir<ST, 3, FF, PART>(k, f, gb, g, cell, fsum, ofeqsum);
  collide_dir<ST, 4, FF, PART>(k, f, gb, g, cell, fsum, ofeqsum);
  collide_dir<ST, 5, FF, PART>(k, f, gb, g, cell, fsum, ofeqsum);
  collide_dir<ST, 6, FF, PART>(k, f, gb, g, cell, fsum, ofeqsum);
  collide_dir<ST, 7, FF, PART>(k, f, gb, g, cell, fsum, ofeqsum);
  collide_dir<ST, 8, FF, PART>(k, f, gb, g, cell, fsum, ofeqsum);
  // f_0 = phi - sum_{a>0} f_a and omega_f (f_0^eq - f_0) = omega_f sum_{a>0} f_a - sum omega_f f^eq_a;
  // the directions a > 0 carry w_a phiD of the source inside ofeqsum, so the rest gets
  // phiD - (5/9) phiD = w_0 phiD by adding phiD:
  // f*_0 = phi_hi + [(phi_lo - sum f_a) + (omega_f sum f_a - sum (omega_f f^eq_a + w_a phiD)) + phiD].
  // Only small terms are rounded before the one error-free sum with the O(1) high word.
  if (PART == COLLIDE_G) return;
  fsum = to_scale<ST>(fsum, g.isf);          // back from the storage scale (exact)
  ofeqsum = to_scale<ST>(ofeqsum, g.isf);
  float hi, lo;
  if constexpr (FF) {
    // the forced form changes phi by theta_M lap mu (+ phiD) in the collision
    two_sum(phi_hi, fadd(fadd(fadd(fsub(phi_lo, fsum), fmad(P.omega_f, fsum, -ofeqsum)), fmul(P.thM6, r.lmu6)), phiD),
            hi, lo);
  } else {
    two_sum(phi_hi, fadd(fadd(fsub(phi_lo, fsum), fmad(P.omega_f, fsum, -ofeqsum)), phiD), hi, lo);
  }
  if (ST == ST_FP32) {
    st_pop<ST>(g.dst, 0, cell, hi, 1.0f);
    st_pop<ST>(g.dst, PLANE_F0LO, cell, lo, 1.0f);
  } else {
    st_pop<ST>(g.dst, 0, cell, fadd(hi, lo), 1.0f);
  }
}

// ---- Per-cell stage arithmetic, shared by every step kernel (the row march below and the 2-D
// tile kernel), so that a cell's result does not depend on the kernel that computes it.  Stencil
// arguments point at the cell's column in rows s (south), 0 and n (north); [-1] and [1] are the
// west and east neighbours.

// S0: phi = sum_a f_a as an unevaluated pair hi + lo (fp[0..8] f_0..f_8, fp[9] f_0lo).
// fp[1..8] in storage scale (isf: its inverse).
template <int ST>
__device__ __forceinline__ void phi_pair(const float fp[NF], float isf, float& hi, float& lo) {
  const float s8 = fadd(fadd(fadd(fp[1], fp[2]), fadd(fp[3], fp[4])), fadd(fadd(fp[5], fp[6]), fadd(fp[7], fp[8])));
  const float small = fadd(fp[Q], to_scale<ST>(s8, isf));
  two_sum(fp[0], small, hi, lo);
}

// S1: mu = theta'(phi) - kappa lap(phi) (Eq. 1) from the phi pair's 3x3 neighbourhood.
__device__ __forceinline__ float chem_potential(const Phys& P, const float* hs, const float* h0, const float* hn,
                                               const float* ls, const float* l0, const float* ln) {
  const float H = h0[0], L = l0[0];
  // differences from the centre: exact for neighbouring values of like magnitude; the low
  // words are tiny and are summed directly
  const float dax = fadd(fadd(fsub(h0[1], H), fsub(hn[0], H)), fadd(fsub(h0[-1], H), fsub(hs[0], H)));
  const float ddg = fadd(fadd(fsub(hn[1], H), fsub(hn[-1], H)), fadd(fsub(hs[-1], H), fsub(hs[1], H)));
  const float lax = fadd(fadd(l0[1], ln[0]), fadd(l0[-1], ls[0]));
  const float ldg = fadd(fadd(ln[1], ln[-1]), fadd(ls[-1], ls[1]));
  const float lap6 = fmad(-20.0f, L, fmad(4.0f, fadd(dax, lax), fadd(ddg, ldg)));   // 6 lap(phi)
  const float ph = fadd(H, L);
  const float dm = fadd(fsub(H, P.phi_star), L), dp = fadd(fadd(H, P.phi_star), L);
  return fmad(-P.kappa6, lap6, fmul(fmul(fmul(P.four_beta, ph), dm), dp));
}

// 6 lap(q) of the isotropic 9-point Laplacian.
__device__ __forceinline__ float lap6_of(const float* s, const float* c, const float* n) {
  return fmad(-20.0f, c[0], fmad(4.0f, fadd(fadd(c[1], n[0]), fadd(c[-1], s[0])), fadd(fadd(n[1], n[-1]), fadd(s[-1], s[1]))));
}

// S2: density, surface and body forces, velocity (the second-order scheme of Eq. 8, F_a removed
// or not) and pressure of a cell from phi, 12 grad(phi), 12 grad(mu), mu, the mass defect s and
// the pulled gbar populations.
struct S2Out {
  float rho, cl, fsx, fsy, gy, rrho, ux, uy, rx, ry, p;
};
// gb[] in storage scale (isg: its inverse).
template <int ST>
__device__ __forceinline__ S2Out s2_cell(const Phys& P, float ph, float gphx, float gphy, float gmx, float gmy,
                                         float mu0, float sdef, const float gb[Q], float isg) {
  S2Out o;
  o.cl = __saturatef(fmad(ph, P.inv_2phistar, 0.5f));   // clamp((phi + phi*) / (2 phi*))
  o.rho = fmad(o.cl, P.drho, P.rho_B);
  if (P.fs_mu) {                                        // F_s = mu grad phi, or -phi grad mu
    const float mu12 = fmul(mu0, 1.0f / 12.0f);
    o.fsx = fmul(mu12, gphx);
    o.fsy = fmul(mu12, gphy);
  } else {
    const float mph12 = fmul(ph, -1.0f / 12.0f);
    o.fsx = fmul(mph12, gmx);
    o.fsy = fmul(mph12, gmy);
  }
  o.gy = fmul(-P.gravity, o.rho);
  const float s13 = fadd(gb[1], gb[3]), d13 = fsub(gb[1], gb[3]);
  const float s24 = fadd(gb[2], gb[4]), d24 = fsub(gb[2], gb[4]);
  const float s57 = fadd(gb[5], gb[7]), d57 = fsub(gb[5], gb[7]);
  const float s68 = fadd(gb[6], gb[8]), d86 = fsub(gb[8], gb[6]);
  const float m0g = to_scale<ST>(fadd(fadd(fadd(gb[0], s13), fadd(s24, s57)), s68), isg);
  const float jx = to_scale<ST>(fadd(fadd(d13, d57), d86), isg);
  const float jy = to_scale<ST>(fsub(fadd(d24, d57), d86), isg);
  o.rrho = __fdividef(1.0f, o.rho);
  const float rden = P.remove_Fa ? __fdividef(1.0f, fmad(-0.5f, sdef, o.rho)) : o.rrho;
  o.ux = fmul(fmad(3.0f, jx, fmul(0.5f, o.fsx)), rden);
  o.uy = fmul(fmad(3.0f, jy, fmul(0.5f, fadd(o.fsy, o.gy))), rden);
  o.rx = fmul(P.rho_prime12, gphx);                     // grad rho
  o.ry = fmul(P.rho_prime12, gphy);
  o.p = fmad(fmad(o.ux, o.rx, fmul(o.uy, o.ry)), 1.0f / 6.0f, m0g);
  return o;
}

// The record S3 needs from S2 (the forced order-parameter fields are set by the caller).
__device__ __forceinline__ void s2_record(const Phys& P, const S2Out& o, float ph, float mu0, float sdef, Rec& r) {
  r.phi = ph;
  r.mu = mu0;
  r.ux = o.ux;
  r.uy = o.uy;
  r.Fx = P.remove_Fa ? fmad(o.ux, sdef, o.fsx) : o.fsx;
  r.Fy = P.remove_Fa ? fmad(o.uy, sdef, fadd(o.fsy, o.gy)) : fadd(o.fsy, o.gy);
  r.mrx3 = fmul(-1.0f / 3.0f, o.rx);
  r.mry3 = fmul(-1.0f / 3.0f, o.ry);
  const float muv3 = fmad(o.cl, P.mu3_d, P.mu3_B);      // 3 mu(phi)
  r.og = __fdividef(1.0f, fmad(muv3, o.rrho, 0.5f));    // 1 / tau_g(phi)
  r.ogr3 = fmul(r.og, fmul(o.rho, 1.0f / 3.0f));
}

// S3: phi div(u) of the convective Cahn-Hilliard source from u_x rows (xs, x0, xn) and u_y rows
// (ys, yn): 12 d(ux)/dx = 4 (E - W) + (NE - SW) - (NW - SE), 12 d(uy)/dy = 4 (N - S) + (NE - SW) + (NW - SE).
__device__ __forceinline__ float phi_div_u(float phi, const float* xs, const float* x0, const float* xn, const float* ys,
                                           const float* yn) {
  const float dux = fmad(4.0f, fsub(x0[1], x0[-1]), fsub(fsub(xn[1], xs[-1]), fsub(xn[-1], xs[1])));
  const float duy = fmad(4.0f, fsub(yn[0], ys[0]), fadd(fsub(yn[1], ys[-1]), fsub(yn[-1], ys[1])));
  return fmul(phi, fmul(fadd(dux, duy), 1.0f / 12.0f));
}

// The fused step (MODE_STEP) or the moment evaluation (MODE_MOMENTS) over one tile:
// columns [x0, x0 + tile_w) x rows [ya, yb) of one simulation.
//
// Stencils read fixed neighbours (t +- 1, row +- 1) of the shared rings.  Beyond a wall the
// ghost value is the mirror image of the first/last row or column (zero normal gradient); the
// thread that computes a value next to a wall also stores it into that ghost slot, so no read
// is remapped.  Only one ghost row/column is ever read because every stage runs on real cells
// and the stencils have radius 1.
// Inlined into both kernels; its arithmetic is fixed by the explicit intrinsics above.
// SD: the direct mass defect (s_form 1) is compiled in; kernels without it carry none of its code.
// FF: the forced order-parameter LBE (f_form 1; FP32 storage only).
// XW: the x axis may have walls; false (a periodic x axis) compiles out the ghost columns and the
// column wall tests of the gathers.
// GREG: the pulled gbar of a row stays in registers from S2 to the next iteration's S3 (c3: 41.6
// -> 40.8 us at 149 registers); without it, in a shared-memory slot (the batch kernel, which
// holds 128 registers and would spill).
template <int NT, int MODE, int ST, bool SD, bool FF = false, bool XW = true, bool GREG = true>
__device__ __forceinline__ void run_tile(const Phys P, const Grid g, const MomentOut mo, int strip, int seg,
                                      Smem<NT>& sm) {
  const int t = threadIdx.x;
  const int x0 = strip * g.tile_w;
  const int x_end = min(x0 + g.tile_w, g.nx);
  const int width = x_end - x0;
  const int ya = seg * g.seg_h;
  const int yb = min(ya + g.seg_h, g.ny);
  const int xl = x0 - 3 + t;                 // logical column (may lie outside [0, nx))
  const bool xwall = XW && g.bc_x == BC_WALL;
  const bool ywall = g.bc_y == BC_WALL;
  const bool col_real = !xwall || (xl >= 0 && xl < g.nx);
  const int xp = wrap1(xl, g.nx);
  const bool in_w3 = t < width + 6 && col_real;
  const bool in_w2 = t >= 1 && t < width + 5 && col_real;
  const bool in_w1 = t >= 2 && t < width + 4 && col_real;
  const bool in_w0 = t >= 3 && t < width + 3;
  // ghost column this thread also fills (its mirror image beyond a wall), or -1; a ghost that
  // falls outside the ring (the strip ends 3 columns short of the right wall) is never read
  const int tg = (xwall && xl == 0) ? t - 1 : ((xwall && xl == g.nx - 1 && t + 1 < NT) ? t + 1 : -1);
  const bool has_tg = tg >= 0;
  constexpr int SLOT = R_FIELDS * NT;        // floats per ring slot
  constexpr int RMASK = RING * SLOT - 1;     // ring size is a power of two
  float* const ring = &sm.rows[0][0][0];
  // slot offset (in floats) of row r; rows are consecutive integers, so offsets wrap
  auto slot = [&](int r) { return (r * SLOT) & RMASK; };
  // ghost row beyond a wall filled together with real row r (its mirror), as a slot offset
  auto ghost_slot = [&](int r) { return r == 0 ? slot(-1) : slot(g.ny); };
  // A segment whose touched rows (ya - 9 .. yb + 6, over its whole march) are all interior
  // needs none of the wrap and wall handling in its checked iterations, only the stage tests.
  const bool seg_interior = ya >= 9 && yb + 6 <= g.ny - 1;
  auto is_wall_row = [&](int r) { return !seg_interior && ywall && (r == 0 || r == g.ny - 1); };
  auto row_ok = [&](int r) { return seg_interior || !ywall || (r >= 0 && r < g.ny); };
  ColNb cn = make_col<ST>(xp, g);
  if constexpr (!XW) cn.wl = cn.wr = false;
  constexpr int USLOT = 2 * NT;
  float* const uring = &sm.urows[0][0][0];
  // Ring slot of row r; the ghost rows beyond a wall (-1, ny) have slots of their own, since a
  // 4-row ring would put the top one on a row that S3 of the previous iteration still reads.
  auto uslot = [&](int r) { return (r & (RING_U - 1)) * USLOT; };
  auto uslot_ck = [&](int r) {
    if (seg_interior) return uslot(r);
    return ywall && r < 0 ? RING_U * USLOT : (ywall && r >= g.ny ? (RING_U + 1) * USLOT : uslot(r));
  };

  const int tgi = has_tg ? tg : t;           // ghost target, own column when there is none
  using Checked = std::true_type;            // rows may wrap, lie beyond a wall or be wall rows
  using Inner = std::false_type;             // every touched row is interior (no checks)

  // store field F of row r (slot offset so) plus its mirrored ghost copies
  auto put = [&](int so, int r, int F, float v, auto checked) {
    ring[so + F * NT + t] = v;
    if constexpr (XW) ring[so + F * NT + tgi] = v;   // a second store to the own column when no ghost
    if constexpr (decltype(checked)::value) {
      if (is_wall_row(r)) {
        const int gs = ghost_slot(r);
        ring[gs + F * NT + t] = v;
        if constexpr (XW) ring[gs + F * NT + tgi] = v;
      }
    }
  };

  // u_x, u_y of row r with the same mirrored ghost copies
  auto put_u = [&](int r, float ux, float uy, auto checked) {
    const int so = uslot(r);
    uring[so + t] = ux;
    uring[so + NT + t] = uy;
    if constexpr (XW) {
      uring[so + tgi] = ux;
      uring[so + NT + tgi] = uy;
    }
    if constexpr (decltype(checked)::value) {
      if (is_wall_row(r)) {
        const int gs = r == 0 ? RING_U * USLOT : (RING_U + 1) * USLOT;
        uring[gs + t] = ux;
        uring[gs + NT + t] = uy;
        if constexpr (XW) {
          uring[gs + tgi] = ux;
          uring[gs + NT + tgi] = uy;
        }
      }
    }
  };

  // prefetched gathers (stored bits): f (+ f_0lo) of the next S0 row, gbar of the next S2 row
  unsigned int fpr[NF], gpr[Q];
  unsigned int spr[2];                       // direct mass defect: rho, div(rho u) of the last step
  auto row_nb = [&](int r, auto checked) {
    RowNb rn;
    if constexpr (decltype(checked)::value) {
      if (!seg_interior) return make_row(wrap1(r, g.ny), g);
    }
    rn.r0 = r * g.pitch;
    rn.rm = rn.r0 - g.pitch;
    rn.rq = rn.r0 + g.pitch;
    rn.b0 = r * g.row_bytes;
    rn.bm = rn.b0 - g.row_bytes;
    rn.bq = rn.b0 + g.row_bytes;
    rn.wb = rn.wt = false;
    return rn;
  };
  auto fetch_f = [&](int r, auto checked) {
    const RowNb rn = row_nb(r, checked);
    gather9<ST, 0>(g.src, cn, rn, fpr);
    fpr[Q] = ST == ST_FP32 ? ld_raw<ST>(g.src, PLANE_F0LO, cell_at(rn.b0, cn.c0)) : 0u;
  };
  auto fetch_g = [&](int r, auto checked) {
    const RowNb rn = row_nb(r, checked);
    gather9<ST, Q>(g.src, cn, rn, gpr);
    if constexpr (SD) {
      const float* sp = reinterpret_cast<const float*>(static_cast<const char*>(g.src) + g.spoff);
      spr[0] = __float_as_uint(__ldg(sp + rn.r0 + cn.x0));
      spr[1] = __float_as_uint(__ldg(sp + g.plane + rn.r0 + cn.x0));
    }
  };
  auto s0_active = [&](int r) { return r <= yb + 2 && in_w3 && row_ok(r); };
  auto s2_active = [&](int r) { return r >= ya - 1 && r <= yb && in_w1 && row_ok(r); };
  if (s0_active(ya - 3)) fetch_f(ya - 3, Checked{});

  Rec cur{}, prev{};
  float gcur[Q], gprev[Q];                   // pulled gbar of the S2 row, then of the S3 row
  int fslot = 0;                             // (a - ya + 3) mod RING_F: ring slot of row a
  // One row iteration.  Inner iterations (every stage active, every touched row interior) drop
  // all row tests; the fetches then run for every thread (their columns are always in range).
  auto iter = [&](int a, auto inner_tag) {
    constexpr bool IN = !decltype(inner_tag)::value;
    using CK = decltype(inner_tag);
    // slot offsets of the rows this iteration touches (a-6 .. a)
    const int o0 = slot(a), o1 = slot(a - 1), o2 = slot(a - 2), o3 = slot(a - 3);
    const int o4 = slot(a - 4), o5 = slot(a - 5), o6 = slot(a - 6);
    // ---- S0: phi at row a (as an unevaluated pair hi + lo)
    if (IN ? in_w3 : s0_active(a)) {
      float fp[NF];
#pragma unroll
      for (int k = 0; k < Q; ++k) fp[k] = dec_pop<ST>(fpr[k], k);
      fp[Q] = __uint_as_float(fpr[Q]);
      float hi, lo;
      phi_pair<ST>(fp, g.isf, hi, lo);
      put(o0, a, R_PHI_HI, hi, CK{});
      put(o0, a, R_PHI_LO, lo, CK{});
      if (MODE == MODE_STEP && in_w0 && (IN || a >= ya)) {
#pragma unroll
        for (int k = 0; k < NFR / 2; ++k) sm.f[fslot][t][k] = make_float2(fp[2 * k + 1], fp[2 * k + 2]);
      }
    }
    if (IN || s0_active(a + 1)) fetch_f(a + 1, CK{});
    // ---- S1: mu at row a-2 (rows a-3 .. a-1 of phi)
    {
      const int r = a - 2;
      if (IN ? in_w2 : (r >= ya - 2 && r <= yb + 1 && in_w2 && row_ok(r))) {
        const float* hs = ring + o3 + R_PHI_HI * NT + t;
        const float* h0 = ring + o2 + R_PHI_HI * NT + t;
        const float* hn = ring + o1 + R_PHI_HI * NT + t;
        const float* ls = ring + o3 + R_PHI_LO * NT + t;
        const float* l0 = ring + o2 + R_PHI_LO * NT + t;
        const float* ln = ring + o1 + R_PHI_LO * NT + t;
        put(o2, r, R_MU, chem_potential(P, hs, h0, hn, ls, l0, ln), CK{});
      }
    }
    // ---- S2: u, p at row a-4 (rows a-5 .. a-3 of phi and mu)
    {
      const int r = a - 4;
      if (IN ? in_w1 : s2_active(r)) {
        const float* hs = ring + o5 + R_PHI_HI * NT + t;
        const float* h0 = ring + o4 + R_PHI_HI * NT + t;
        const float* hn = ring + o3 + R_PHI_HI * NT + t;
        const float* ms = ring + o5 + R_MU * NT + t;
        const float* m0 = ring + o4 + R_MU * NT + t;
        const float* mn = ring + o3 + R_MU * NT + t;
        // grad phi only feeds grad rho (density and pressure terms): the high words suffice
        const float ph = fadd(h0[0], ring[o4 + R_PHI_LO * NT + t]);
        float gphx, gphy, gmx, gmy;                // 12 x the isotropic gradients
        grad12(hs, h0, hn, gphx, gphy);
        grad12(ms, m0, mn, gmx, gmy);
        // cell index of row r for the direct mass defect's planes (periodic halo rows wrap)
        auto cell_of = [&]() { return (IN || seg_interior ? r : wrap1(r, g.ny)) * g.pitch + xp; };
        float sdef = 0.0f;
        if (P.remove_Fa || (MODE == MODE_MOMENTS && mo.fax)) {
          if constexpr (SD) {
            // this cell's rho (formed as s2_cell forms it) less the prefetched rho of the last step
            const float rho_ = fmad(__saturatef(fmad(ph, P.inv_2phistar, 0.5f)), P.drho, P.rho_B);
            sdef = fadd(fsub(rho_, __uint_as_float(spr[0])), __uint_as_float(spr[1]));
          } else {
            sdef = fmul(P.s_coef6, lap6_of(ms, m0, mn));
          }
        }
        float gb[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) gb[k] = dec_pop<ST>(gpr[k], Q + k);
        const S2Out s2 = s2_cell<ST>(P, ph, gphx, gphy, gmx, gmy, m0[0], sdef, gb, g.isg);
        const float rho = s2.rho, ux = s2.ux, uy = s2.uy, p = s2.p;
        put(o4, r, R_P, p, CK{});
        if (MODE == MODE_STEP && (P.ch_conv || SD)) put_u(r, ux, uy, CK{});
        if (MODE == MODE_STEP && SD) {
          if (in_w0 && (IN || (r >= ya && r < yb)))
            reinterpret_cast<float*>(static_cast<char*>(g.dst) + g.spoff)[cell_of()] = rho;   // rho^t for the next step
        }
        if (MODE == MODE_MOMENTS) {
          if (in_w0 && (IN || (r >= ya && r < yb))) {
            const int o = r * g.pitch + xp;
            if (mo.phi) mo.phi[o] = ph;
            if (mo.rho) mo.rho[o] = rho;
            if (mo.ux) mo.ux[o] = ux;
            if (mo.uy) mo.uy[o] = uy;
            if (mo.p) mo.p[o] = p;
            if (mo.fax) {
              mo.fax[o] = fmul(-ux, sdef);
              mo.fay[o] = fmul(-uy, sdef);
            }
          }
        } else {
          if (in_w0 && (IN || r >= ya)) {
#pragma unroll
            for (int k = 0; k < Q; ++k) {
              if constexpr (GREG) gcur[k] = gb[k];
              else sm.g[r & 1][k][t] = gb[k];
            }
          }
          s2_record(P, s2, ph, m0[0], sdef, cur);
          if constexpr (FF) {
            cur.gx12 = gphx;
            cur.gy12 = gphy;
            cur.lmu6 = lap6_of(ms, m0, mn);
          }
        }
      }
      if (IN || s2_active(r + 1)) fetch_g(r + 1, CK{});
    }
    __syncthreads();
    // ---- S3: collide and store row a-5 (p of rows a-6 .. a-4)
    if (MODE == MODE_STEP) {
      const int r = a - 5;
      if (IN ? in_w0 : (r >= ya && r < yb && in_w0)) {
        const float* qs = ring + o6 + R_P * NT + t;
        const float* q0 = ring + o5 + R_P * NT + t;
        const float* qn = ring + o4 + R_P * NT + t;
        float gpx, gpy;                          // 12 grad p
        grad12(qs, q0, qn, gpx, gpy);
        float phiD = 0.0f;                       // phi div(u) of the convective form
        if (P.ch_conv) {
          const float* xs_ = uring + (IN ? uslot(a - 6) : uslot_ck(a - 6)) + t;
          const float* x0_ = uring + uslot(a - 5) + t;
          const float* xn_ = uring + (IN ? uslot(a - 4) : uslot_ck(a - 4)) + t;
          phiD = phi_div_u(prev.phi, xs_, x0_, xn_, xs_ + NT, xn_ + NT);
        }
        const int rslot = fslot == RING_F - 1 ? 0 : fslot + 1;   // row a-5 == row a+1 (mod 6)
        float f[Q], gb[Q];
        f[0] = 0.0f;   // unused: f_0 follows from the phi pair
#pragma unroll
        for (int k = 0; k < NFR / 2; ++k) {
          const float2 v = sm.f[rslot][t][k];
          f[2 * k + 1] = v.x;
          f[2 * k + 2] = v.y;
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) gb[k] = GREG ? gprev[k] : sm.g[r & 1][k][t];
        if (SD) {
          // div(rho u) of this step, for the next step's mass defect; rho from the phi rings as in S2
          const float* xs_ = uring + (IN ? uslot(a - 6) : uslot_ck(a - 6)) + t;
          const float* x0_ = uring + uslot(a - 5) + t;
          const float* xn_ = uring + (IN ? uslot(a - 4) : uslot_ck(a - 4)) + t;
          auto rho_at = [&](int o, int dc) {
            const float ph_ = fadd(ring[o + R_PHI_HI * NT + t + dc], ring[o + R_PHI_LO * NT + t + dc]);
            return fmad(__saturatef(fmad(ph_, P.inv_2phistar, 0.5f)), P.drho, P.rho_B);
          };
          const float rE = rho_at(o5, 1), rW = rho_at(o5, -1), rN = rho_at(o4, 0), rS = rho_at(o6, 0);
          const float rNE = rho_at(o4, 1), rNW = rho_at(o4, -1), rSE = rho_at(o6, 1), rSW = rho_at(o6, -1);
          const float jxE = fmul(rE, x0_[1]), jxW = fmul(rW, x0_[-1]);
          const float jxNE = fmul(rNE, xn_[1]), jxNW = fmul(rNW, xn_[-1]), jxSE = fmul(rSE, xs_[1]), jxSW = fmul(rSW, xs_[-1]);
          const float jyN = fmul(rN, xn_[NT]), jyS = fmul(rS, xs_[NT]);
          const float jyNE = fmul(rNE, xn_[NT + 1]), jyNW = fmul(rNW, xn_[NT - 1]);
          const float jySE = fmul(rSE, xs_[NT + 1]), jySW = fmul(rSW, xs_[NT - 1]);
          const float djx = fmad(4.0f, fsub(jxE, jxW), fsub(fsub(jxNE, jxSW), fsub(jxNW, jxSE)));
          const float djy = fmad(4.0f, fsub(jyN, jyS), fadd(fsub(jyNE, jySW), fsub(jyNW, jySE)));
          float* sp = reinterpret_cast<float*>(static_cast<char*>(g.dst) + g.spoff);
          sp[g.plane + r * g.pitch + xp] = fmul(fadd(djx, djy), 1.0f / 12.0f);
        }
        collide_store<ST, FF>(P, prev, q0[0], gpx, gpy, ring[o5 + R_PHI_HI * NT + t], ring[o5 + R_PHI_LO * NT + t], phiD,
                          f, gb, g, cell_at(r * g.row_bytes, cn.c0));
      }
    }
    prev = cur;
    if constexpr (GREG) {
#pragma unroll
      for (int k = 0; k < Q; ++k) gprev[k] = gcur[k];
    }
    fslot = fslot == RING_F - 1 ? 0 : fslot + 1;
  };

  // Inner iterations: all stages active (a in [ya+5, yb+1]) and the rows touched, a-6 .. a+2,
  // interior: no wrap, no wall row, no row beyond a wall (a - 6 >= 0 keeps the u ring's own
  // ghost slots out of inner iterations).
  const int a_in0 = max(ya + 5, 6), a_in1 = min(yb + 1, g.ny - 3);
  int a = ya - 3;
  for (; a <= yb + 4 && a < a_in0; ++a) iter(a, Checked{});
  for (; a <= a_in1; ++a) iter(a, Inner{});
  for (; a <= yb + 4; ++a) iter(a, Checked{});
}

}  // namespace lbm
