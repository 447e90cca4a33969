// Ragged batches: many independent simulations (any sizes and parameters) advanced by one
// persistent launch per time step over a work list of (simulation, strip, segment) tiles; two
// launches when some members use the direct mass defect (its tiles run in their own kernel
// instance).  Steps run as replays of one 16-step CUDA graph captured once per membership, the
// remainder of a step count as direct launches.  Each tile runs exactly the per-cell arithmetic of the single-simulation kernel
// (every operation an explicit round-to-nearest intrinsic), so a member's state is bitwise the
// same alone or inside any mix.
#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "lbm_internal.h"

namespace lbm {

struct SimDesc {
  Phys P;
  Grid g;                 // src/dst unused; buffers below
  const void* buf0;
  void* buf1;
  int cur0;               // buffer holding the state when the graph replay starts
  int pad;
};

// SD: the work list holds the tiles of members that use the direct mass defect (s_form 1), and
// only that tile body is compiled in.  One function holding both bodies (each for three
// storages) did not fit 128 registers: it spilled 1.2 KB per thread, and a batch of s_form 1
// members ran at 14.5 GLUPS against 18.8 with the instances split.
// XW: some member may have walls on x; false compiles out the ghost columns and column wall tests
// (every member periodic in x).
template <int NT, bool SD, bool XW>
__global__ void __launch_bounds__(NT, 512 / NT) k_batch(const SimDesc* __restrict__ sims, const int4* __restrict__ work,
                                              int n_work, int parity) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<NT>& sm = *reinterpret_cast<Smem<NT>*>(smem_raw);
  for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
    const int4 it = work[w];
    const SimDesc& d = sims[it.x];
    Grid g = d.g;
    const bool odd = ((d.cur0 + parity) & 1) != 0;
    g.src = odd ? d.buf1 : d.buf0;
    g.dst = odd ? const_cast<void*>(d.buf0) : d.buf1;
    // members may differ in storage; the branch is uniform per tile
    switch (g.storage) {
      case ST_FP16: run_tile<NT, MODE_STEP, ST_FP16, SD, false, XW, false>(d.P, g, MomentOut{}, it.y, it.z, sm); break;
      case ST_BF16: run_tile<NT, MODE_STEP, ST_BF16, SD, false, XW, false>(d.P, g, MomentOut{}, it.y, it.z, sm); break;
      default: run_tile<NT, MODE_STEP, ST_FP32, SD, false, XW, false>(d.P, g, MomentOut{}, it.y, it.z, sm); break;
    }
    __syncthreads();  // shared rings are reused by the next tile
  }
}

}  // namespace lbm

using namespace lbm;

template <bool SD, bool XW>
static cudaError_t set_batch_attr_sd(int nt) {
  switch (nt) {
    case 64: return cudaFuncSetAttribute(k_batch<64, SD, XW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<64>));
    case 256: return cudaFuncSetAttribute(k_batch<256, SD, XW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<256>));
    default: return cudaFuncSetAttribute(k_batch<128, SD, XW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<128>));
  }
}

// Members with the direct mass defect always run the general form: its periodic form does not
// fit 128 registers (it spilled 36 bytes per thread).
static cudaError_t set_batch_attr(int nt, bool sd, bool xw) {
  if (sd) return set_batch_attr_sd<true, true>(nt);
  return xw ? set_batch_attr_sd<false, true>(nt) : set_batch_attr_sd<false, false>(nt);
}

template <bool SD, bool XW>
static int batch_occupancy_t(int nt) {
  int occ = 0;
  switch (nt) {
    case 64: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<64, SD, XW>, 64, sizeof(Smem<64>)); break;
    case 256: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<256, SD, XW>, 256, sizeof(Smem<256>)); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<128, SD, XW>, 128, sizeof(Smem<128>)); break;
  }
  return occ;
}

template <bool SD>
static int batch_occupancy_sd(int nt, bool xw) {
  if constexpr (SD) return batch_occupancy_t<SD, true>(nt);
  else return xw ? batch_occupancy_t<SD, true>(nt) : batch_occupancy_t<SD, false>(nt);
}

constexpr int GRAPH_STEPS = 16;        // steps per captured graph (even: parity-neutral)

struct lbm_batch {
  size_t budget = 0;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;          // private stream for graph capture
  std::vector<lbm_sim*> slots;         // nullptr = free slot
  int nt = 128;
  int seg_h = 32;                      // rows per tile for members without their own choice
  bool dirty = true;                   // descriptors / work list need rebuilding
  SimDesc* d_sims = nullptr;
  int4* d_work = nullptr;
  size_t cap_sims = 0, cap_work = 0;
  int n_work = 0;
  int n_plain = 0;                     // work[0, n_plain): members without the direct mass defect
  int grid_plain = 0, grid_sd = 0;     // persistent grid of each launch
  int flip = 0;                        // parity offset of every member since the last rebuild
  bool xwall = true;                   // some member has walls on x (the general kernel form)
  std::map<int, cudaGraphExec_t> graphs;  // flip -> executable graph of GRAPH_STEPS steps
};

static void drop_graphs(lbm_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

static int rebuild(lbm_batch* b) {
  std::vector<SimDesc> sims;
  std::vector<int4> work;
  std::vector<int> members;
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (b->slots[i]) members.push_back((int)i);
  // interleave the members' tiles so concurrent CTAs spread over simulations; the tiles of
  // members with the direct mass defect follow those of the others (a launch of their own)
  std::vector<std::vector<int4>> per[2];
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->xwall = false;
  for (int m : members) b->xwall = b->xwall || b->slots[m]->params.bc_x == LBM_WALL;
  set_batch_attr(b->nt, false, b->xwall);   // the occupancy query needs the shared-memory size admitted
  const int slots = sms * std::max(batch_occupancy_sd<false>(b->nt, b->xwall), 1);
  for (size_t m = 0; m < members.size(); ++m) {
    lbm_sim* s = b->slots[members[m]];
    SimDesc d{};
    d.P = s->phys;
    Grid g = make_grid(s, nullptr, nullptr);
    // one wave of the batch kernel is shared by all members: size segments for the batch.  A
    // member large enough to fill the wave on its own gets segments of the height that does so
    // (as a simulation stepped alone): fewer, taller tiles cut its pipeline-fill rows.
    int h = s->seg_h ? s->seg_h : b->seg_h;
    if (!s->seg_h) {
      int tw = 0, ns = 0, hw = 0;
      tile_geometry(s->nx, s->ny, b->nt, 0, slots, &tw, &ns, &hw);
      h = std::max(h, hw);
    }
    tile_geometry(s->nx, s->ny, b->nt, h, 0, &g.tile_w, &g.n_strips, &g.seg_h);
    d.g = g;
    d.buf0 = s->buf[0];
    d.buf1 = s->buf[1];
    d.cur0 = s->cur;
    sims.push_back(d);
    std::vector<int4> tl;
    const int nseg = (s->ny + g.seg_h - 1) / g.seg_h;
    for (int sg = 0; sg < nseg; ++sg)
      for (int st = 0; st < g.n_strips; ++st) tl.push_back(make_int4((int)m, st, sg, 0));
    per[d.P.s_direct ? 1 : 0].push_back(std::move(tl));
  }
  int n_plain = 0;
  for (int part = 0; part < 2; ++part) {
    size_t most = 0;
    for (auto& v : per[part]) most = std::max(most, v.size());
    for (size_t k = 0; k < most; ++k)
      for (auto& v : per[part])
        if (k < v.size()) work.push_back(v[k]);
    if (part == 0) n_plain = (int)work.size();
  }
  cudaError_t e;
  if (sims.size() > b->cap_sims) {
    cudaFree(b->d_sims);
    b->d_sims = nullptr;
    b->cap_sims = 0;
    if ((e = cudaMalloc(&b->d_sims, sims.size() * sizeof(SimDesc))) != cudaSuccess) return cuda_fail(e, "batch descriptors");
    b->cap_sims = sims.size();
  }
  if (work.size() > b->cap_work) {
    cudaFree(b->d_work);
    b->d_work = nullptr;
    b->cap_work = 0;
    if ((e = cudaMalloc(&b->d_work, work.size() * sizeof(int4))) != cudaSuccess) return cuda_fail(e, "batch work list");
    b->cap_work = work.size();
  }
  if (!sims.empty() &&
      (e = cudaMemcpyAsync(b->d_sims, sims.data(), sims.size() * sizeof(SimDesc), cudaMemcpyHostToDevice, b->stream)) !=
          cudaSuccess)
    return cuda_fail(e, "batch descriptor upload");
  if (!work.empty() &&
      (e = cudaMemcpyAsync(b->d_work, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream)) !=
          cudaSuccess)
    return cuda_fail(e, "batch work upload");
  // host vectors die here: make the uploads complete first
  if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return cuda_fail(e, "batch upload sync");
  b->n_work = (int)work.size();
  b->n_plain = n_plain;
  b->grid_plain = b->grid_sd = 0;
  if (b->n_plain > 0) {
    if ((e = set_batch_attr(b->nt, false, b->xwall)) != cudaSuccess) return cuda_fail(e, "batch kernel attribute");
    b->grid_plain = std::max(1, std::min(b->n_plain, sms * std::max(batch_occupancy_sd<false>(b->nt, b->xwall), 1)));
  }
  if (b->n_work > b->n_plain) {
    if ((e = set_batch_attr(b->nt, true, b->xwall)) != cudaSuccess) return cuda_fail(e, "batch kernel attribute");
    b->grid_sd = std::max(1, std::min(b->n_work - b->n_plain, sms * std::max(batch_occupancy_sd<true>(b->nt, b->xwall), 1)));
  }
  b->flip = 0;
  drop_graphs(b);
  b->dirty = false;
  return LBM_OK;
}

template <bool SD, bool XW>
static void launch_part_t(lbm_batch* b, const int4* work, int n, int grid, int parity, cudaStream_t st) {
  switch (b->nt) {
    case 64: k_batch<64, SD, XW><<<grid, 64, sizeof(Smem<64>), st>>>(b->d_sims, work, n, parity); break;
    case 256: k_batch<256, SD, XW><<<grid, 256, sizeof(Smem<256>), st>>>(b->d_sims, work, n, parity); break;
    default: k_batch<128, SD, XW><<<grid, 128, sizeof(Smem<128>), st>>>(b->d_sims, work, n, parity); break;
  }
}

template <bool SD>
static void launch_part(lbm_batch* b, const int4* work, int n, int grid, int parity, cudaStream_t st) {
  if constexpr (SD) {
    launch_part_t<SD, true>(b, work, n, grid, parity, st);
  } else {
    if (b->xwall) launch_part_t<SD, true>(b, work, n, grid, parity, st);
    else launch_part_t<SD, false>(b, work, n, grid, parity, st);
  }
}

// One time step of every member: the two launches touch disjoint members.
static cudaError_t launch_batch(lbm_batch* b, int parity, cudaStream_t st) {
  if (b->n_plain > 0) launch_part<false>(b, b->d_work, b->n_plain, b->grid_plain, parity, st);
  if (b->n_work > b->n_plain)
    launch_part<true>(b, b->d_work + b->n_plain, b->n_work - b->n_plain, b->grid_sd, parity, st);
  return cudaGetLastError();
}

extern "C" {

int lbm_batch_create(size_t budget_bytes, void* cuda_stream, lbm_batch** out) {
  if (!out) return set_error("out is NULL"), LBM_ERR_INVALID_ARG;
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return set_error("host allocation failed"), LBM_ERR_OOM;
  b->budget = budget_bytes;
  b->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch stream");
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_add(lbm_batch* b, lbm_sim* s, int* slot) {
  Range range_("lbm_batch_add");
  if (!b || !s) return set_error("batch and sim are required"), LBM_ERR_INVALID_ARG;
  if (s->batch) return set_error("simulation already belongs to a batch"), LBM_ERR_INVALID_ARG;
  if (s->params.f_form)
    return set_error("f_form 1 simulations are stepped alone (the batch kernel has no forced form)"),
           LBM_ERR_INVALID_ARG;
  const size_t need = lbm_sim_device_bytes(s);
  if (b->budget && b->bytes + need > b->budget) {
    set_error("batch budget: %zu + %zu > %zu bytes", b->bytes, need, b->budget);
    return LBM_ERR_BUDGET;
  }
  // the member's earlier work (init, steps) was queued on its own stream
  cudaStreamSynchronize(s->stream);
  int k = -1;
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (!b->slots[i]) {
      k = (int)i;
      break;
    }
  if (k < 0) {
    k = (int)b->slots.size();
    b->slots.push_back(nullptr);
  }
  b->slots[k] = s;
  s->batch = b;
  b->bytes += need;
  b->dirty = true;
  if (slot) *slot = k;
  return LBM_OK;
}

int lbm_batch_remove(lbm_batch* b, int slot) {
  Range range_("lbm_batch_remove");
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot])
    return set_error("invalid batch slot %d", slot), LBM_ERR_INVALID_ARG;
  lbm_sim* s = b->slots[slot];
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch remove sync");
  s->batch = nullptr;
  b->bytes -= lbm_sim_device_bytes(s);
  b->slots[slot] = nullptr;
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int k) {
  Range range_("lbm_batch_step");
  if (!b || k < 0) return set_error("invalid batch or step count"), LBM_ERR_INVALID_ARG;
  if (k == 0) return LBM_OK;
  int rc;
  if (b->dirty && (rc = rebuild(b))) return rc;
  if (b->n_work == 0) return LBM_OK;
  // Whole blocks of GRAPH_STEPS steps replay one graph captured once per membership (the block
  // is even, so a replay leaves the buffer parity as it found it); the remaining k mod
  // GRAPH_STEPS steps are launched directly.  Round lengths then vary freely without a new
  // capture each time.
  const int blocks = k / GRAPH_STEPS, rest = k % GRAPH_STEPS;
  cudaError_t e = cudaSuccess;
  if (blocks > 0) {
    cudaGraphExec_t exec = nullptr;
    auto it = b->graphs.find(b->flip);
    if (it != b->graphs.end()) {
      exec = it->second;
    } else {
      cudaGraph_t graph;
      e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(e, "batch capture begin");
      for (int i = 0; i < GRAPH_STEPS && e == cudaSuccess; ++i) e = launch_batch(b, b->flip + i, b->cap);
      cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
      if (e != cudaSuccess) return cuda_fail(e, "batch capture launch");
      if (e2 != cudaSuccess) return cuda_fail(e2, "batch capture end");
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "batch graph instantiate");
      b->graphs[b->flip] = exec;
    }
    for (int i = 0; i < blocks && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
  }
  for (int i = 0; i < rest && e == cudaSuccess; ++i) e = launch_batch(b, b->flip + i, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch step launch");
  bool flip = (k & 1) != 0;
  for (lbm_sim* s : b->slots) {
    if (!s) continue;
    s->steps += k;
    s->launches += k;
    if (flip) s->cur ^= 1;
  }
  if (flip) b->flip ^= 1;
  return LBM_OK;
}

int lbm_batch_set_tile(lbm_batch* b, int threads, int seg_rows) {
  if (!b) return set_error("batch is NULL"), LBM_ERR_INVALID_ARG;
  if (threads && threads != 64 && threads != 128 && threads != 256)
    return set_error("threads must be 64, 128 or 256"), LBM_ERR_INVALID_ARG;
  if (seg_rows < 0) return set_error("seg_rows must be >= 1"), LBM_ERR_INVALID_ARG;
  if (threads) b->nt = threads;
  if (seg_rows) b->seg_h = seg_rows;
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_size(const lbm_batch* b) {
  if (!b) return 0;
  int n = 0;
  for (lbm_sim* s : b->slots) n += s != nullptr;
  return n;
}

size_t lbm_batch_bytes(const lbm_batch* b) { return b ? b->bytes : 0; }

int lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  cudaStreamSynchronize(b->stream);
  for (lbm_sim* s : b->slots)
    if (s) s->batch = nullptr;
  drop_graphs(b);
  cudaFree(b->d_sims);
  cudaFree(b->d_work);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return LBM_OK;
}

}  // extern "C"
