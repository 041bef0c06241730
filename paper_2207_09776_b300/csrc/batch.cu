// S10: uneven batches (grids 64^2, 128^2, 256^2, any path counts) in one
// persistent launch, captured with the batch's Brownian and weight kernels in
// a CUDA graph, with the work layout chosen by a small autotuner.
//
// The megakernel runs thread-block clusters of four 512-thread CTAs, one CTA
// per SM, and each item's paths in decreasing order of estimated Taylor cost
// (path_order.cu).  Work comes in two kinds, each from its own atomic counter,
// and is run with the engine's per-path solver (engine_core.cuh):
//   units, taken by a whole cluster:
//     D256   one 256^2 path, split into four 64-row slabs (the cluster's CTAs)
//     D128   up to four 128^2 paths, one per CTA
//     D64x2  up to eight 64^2 paths, two per CTA (two 256-thread halves, each
//            synchronised by its own named barrier)
//     D64x1  up to four 64^2 paths, one per CTA (512 threads, two rows each)
//   tasks, taken by one CTA once the units are gone: one 128^2 path, two 64^2
//     paths (one per half) or one 64^2 path, so that no CTA waits for the
//     slowest path of a unit
// Every CTA holds about the same number of grid points (16384) whatever it
// runs, so the work items differ in length only by their Taylor work, which
// grows with the grid (the operator norm scales like 1/Delta^2).
//
// Tuned choices (the "variant"): for 0..3, bit 0 puts every path in units with
// the items interleaved, or (clear) the 256^2 paths in units and the smaller
// grids' paths in tasks, largest grids first; bit 1 packs 64^2 paths two per CTA
// or one per CTA; variant 4 replaces the megakernel by each item's own engine
// launch (its best per-grid configuration) inside the same graph.
// msk_batch_tune times all five on the batch itself and keeps the fastest; the
// result can be cached in a text file keyed by device name and batch shape.
#include <stdio.h>

#include <new>

#include <algorithm>
#include <string>
#include <vector>

#include "engine_core.cuh"

extern const double kMskScaleCap;
msk_status msk_prepare_brownian(msk_ctx* ctx, cudaStream_t stream);
msk_status msk_prepare_omega(msk_ctx* ctx);

namespace {

enum { UNIT_D256 = 0, UNIT_D128 = 1, UNIT_D64X2 = 2, UNIT_D64X1 = 3 };

struct BatchUnit {
  int32_t type, item;
  int64_t first;
  int32_t count, pad;
};

constexpr int kNT = 512;    // threads of a CTA that runs the smaller grids' paths
constexpr int kNT256 = 256;  // threads of a CTA of the clusters that run only 256^2 units
template <int NTB> using K256 = Cfg<float, 256, 4, NTB>;
using K128 = Cfg<float, 128, 1, kNT>;
using K64h = Cfg<float, 64, 1, kNT / 2>;
using K64 = Cfg<float, 64, 1, kNT>;
constexpr size_t kHalf64 = (K64h::SMEM + 255) / 256 * 256;   // byte offset of the second half-slab
constexpr size_t kSmallBytes = std::max(K128::SMEM, std::max(2 * kHalf64, K64::SMEM));
// slab of a megakernel CTA (+ 16 bytes: the unit index slot): with 512 threads it
// runs every unit type, with 256 threads only 256^2 units (partial sum in registers)
template <int NTB> constexpr size_t slab_bytes() {
  return NTB == kNT ? std::max(K256<kNT>::SMEM, kSmallBytes) : K256<NTB>::SMEM;
}
template <int NTB> constexpr size_t batch_smem() { return slab_bytes<NTB>() + 16; }
constexpr size_t kTaskSmem = kSmallBytes + 16;   // + the task index slot
static_assert(batch_smem<kNT>() <= 232448 && batch_smem<kNT256>() <= 232448, "batch slab does not fit shared memory");

// Position pos of an item's cost order -> path index (identity without an order).
__device__ __forceinline__ int64_t path_at(const EngineArgs& a, int64_t pos) { return a.order ? a.order[pos] : pos; }

// The paths of a unit of small grids that fall to CTA `sub` of the cluster, or
// of a task (sub = 0): one 128^2 path, two 64^2 paths (one per 256-thread half)
// or one 64^2 path.
__device__ __forceinline__ void run_small(const BatchUnit& un, const EngineArgs& a, int sub, unsigned char* smem_raw,
                                          int tid) {
  float* sm = reinterpret_cast<float*>(smem_raw);
  switch (un.type) {
    case UNIT_D128: {
      const CtaSync s;
      slab_init<float, 128, 1, kNT>(sm, tid, 0, s);
      if (sub < un.count) solve_path<float, 128, 1, kNT, false>(a, path_at(a, un.first + sub), sm, tid, 0, s);
      break;
    }
    case UNIT_D64X2: {
      const int g = tid / (kNT / 2), t = tid % (kNT / 2);
      const NamedSync s{1 + g, kNT / 2};
      float* half = reinterpret_cast<float*>(smem_raw + g * kHalf64);
      slab_init<float, 64, 1, kNT / 2>(half, t, 0, s);
      const int idx = 2 * sub + g;
      if (idx < un.count) solve_path<float, 64, 1, kNT / 2, false>(a, path_at(a, un.first + idx), half, t, 0, s);
      break;
    }
    default: {
      const CtaSync s;
      slab_init<float, 64, 1, kNT>(sm, tid, 0, s);
      if (sub < un.count) solve_path<float, 64, 1, kNT, false>(a, path_at(a, un.first + sub), sm, tid, 0, s);
      break;
    }
  }
}

// The units, each taken by a whole cluster from counter[0] (NTB = 256: 256^2 units only).
template <int NTB>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(NTB, 1)
    batch_kernel(const EngineArgs* __restrict__ items, const BatchUnit* __restrict__ units, int n_units,
                 unsigned int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  int* s_unit = reinterpret_cast<int*>(smem_raw + slab_bytes<NTB>());
  const int tid = threadIdx.x;
  const int rank = (int)cg::this_cluster().block_rank();
  const ClusterSync csync;
  // every CTA of this grid is resident (one wave of clusters): the task kernel,
  // launched as this kernel's programmatic dependent, may start on the SMs that
  // no cluster of four can use
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (;;) {
    // The previous unit is finished by every CTA once all have reached this
    // barrier; rank 0 then publishes the next unit index in its shared memory.
    if (rank == 0 && tid == 0) *s_unit = (int)atomicAdd(counter, 1u);
    csync();
    const int u = *cg::this_cluster().map_shared_rank(s_unit, 0);
    // Every CTA has read the index before rank 0 may overwrite it or exit
    // (a CTA's shared memory must not be read through DSMEM after it exits).
    csync();
    if (u >= n_units) break;                        // same value in every thread of the cluster
    const BatchUnit un = units[u];
    const EngineArgs a = items[un.item];
    if (un.type == UNIT_D256) {
      slab_init<float, 256, 4, NTB>(sm, tid, rank, csync);
      solve_path<float, 256, 4, NTB, false>(a, path_at(a, un.first), sm, tid, rank, csync);
    } else {
      if constexpr (NTB == kNT) run_small(un, a, rank, smem_raw, tid);
    }
  }
}

// The tasks, each taken by one CTA from counter[1] (no clusters: every SM, and
// a register allocation of its own).  It reads nothing the megakernel writes.
__global__ void __launch_bounds__(kNT, 1)
    batch_task_kernel(const EngineArgs* __restrict__ items, const BatchUnit* __restrict__ tasks, int n_tasks,
                      unsigned int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* s_task = reinterpret_cast<int*>(smem_raw + kSmallBytes);
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) *s_task = (int)atomicAdd(counter + 1, 1u);
    __syncthreads();
    const int q = *s_task;
    __syncthreads();   // read by every thread before thread 0 takes the next one
    if (q >= n_tasks) break;
    const BatchUnit un = tasks[q];
    run_small(un, items[un.item], 0, smem_raw, tid);
  }
}

}  // namespace

struct msk_batch {
  int device = 0;
  std::vector<msk_batch_item> items;
  std::vector<EngineArgs> args;
  std::vector<size_t> f_off, w_off, o_off;   // functionals, weights, path order + queue counter
  std::vector<size_t> p_off;                 // power-norm table of the (s, m) selection (floats)
  double* scratch = nullptr;
  EngineArgs* d_args = nullptr;
  BatchUnit* d_units = nullptr;   // units, then tasks (units_cap entries)
  unsigned int* d_counter = nullptr;   // [0] unit queue, [1] task queue
  int n_units = 0, n_tasks = 0, units_cap = 0;
  int variant = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;   // private stream the graph is captured on
  std::string key;
  std::string err;
};

namespace {

msk_status bfail(msk_batch* b, msk_status st, const std::string& m) {
  if (b) b->err = m;
  return st;
}
msk_status bcuda(msk_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MSK_OK;
  cudaGetLastError();
  return bfail(b, e == cudaErrorMemoryAllocation ? MSK_ERR_OOM : MSK_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

// Variant 4: no megakernel; the graph holds each item's own engine launch.
constexpr int kPerGridVariant = 4;
constexpr int kVariants = 5;

// The work of a megakernel variant: units, each run by a whole cluster, and
// tasks, each run by one CTA.  Positions count along each item's cost order.
//   interleaved (bit 0): every path in units (one 256^2 path, four 128^2 paths,
//     eight or four 64^2 paths), the items' units taken in turn; no tasks
//   longest first: the 256^2 paths as units; the 128^2 paths, then the 64^2
//     ones, as tasks of one path (or two 64^2 paths on the two halves of a CTA),
//     so a CTA waits for no other CTA's path once the 256^2 units are gone
void build_units(const msk_batch* b, int variant, std::vector<BatchUnit>* units, std::vector<BatchUnit>* tasks) {
  const bool interleave = variant & 1, one64 = variant & 2;
  std::vector<std::vector<BatchUnit>> per(b->items.size());
  for (size_t k = 0; k < b->items.size(); ++k) {
    const msk_batch_item& it = b->items[k];
    const int d = it.ctx->d;
    const int type = d == 256 ? UNIT_D256 : d == 128 ? UNIT_D128 : one64 ? UNIT_D64X1 : UNIT_D64X2;
    const int per_cta = type == UNIT_D64X2 ? 2 : 1;
    const int per_unit = type == UNIT_D256 || !interleave ? per_cta : 4 * per_cta;
    for (int64_t p = 0; p < it.paths; p += per_unit)
      per[k].push_back({type, (int32_t)k, p, (int32_t)std::min<int64_t>(per_unit, it.paths - p), 0});
  }
  units->clear();
  tasks->clear();
  if (interleave) {
    for (size_t r = 0;; ++r) {
      bool any = false;
      for (auto& v : per)
        if (r < v.size()) {
          units->push_back(v[r]);
          any = true;
        }
      if (!any) break;
    }
  } else {
    for (auto& v : per)
      for (const BatchUnit& u : v) (u.type == UNIT_D256 ? units : tasks)->push_back(u);
    // larger grids first: they carry more Taylor work per grid point
    std::stable_sort(tasks->begin(), tasks->end(), [&](const BatchUnit& x, const BatchUnit& y) {
      return b->items[x.item].ctx->d > b->items[y.item].ctx->d;
    });
  }
}

void drop_graph(msk_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

msk_status set_variant(msk_batch* b, int variant) {
  std::vector<BatchUnit> units, tasks;
  build_units(b, variant, &units, &tasks);
  const size_t n = units.size() + tasks.size();
  if ((int)n > b->units_cap) {
    if (b->d_units) cudaFree(b->d_units);
    b->d_units = nullptr;
    msk_status st = bcuda(b, cudaMalloc(&b->d_units, std::max<size_t>(1, n) * sizeof(BatchUnit)),
                          "unit list allocation");
    if (st != MSK_OK) return st;
    b->units_cap = (int)n;
  }
  units.insert(units.end(), tasks.begin(), tasks.end());
  if (n > 0) {
    msk_status st = bcuda(b, cudaMemcpy(b->d_units, units.data(), n * sizeof(BatchUnit), cudaMemcpyHostToDevice),
                          "unit list upload");
    if (st != MSK_OK) return st;
  }
  b->n_units = (int)(n - tasks.size());
  b->n_tasks = (int)tasks.size();
  b->variant = variant;
  drop_graph(b);
  return MSK_OK;
}

// Enqueue the whole batch on `s`: counter reset, per-item Brownian functionals,
// weights and path cost order, then the persistent megakernel.
msk_status enqueue(msk_batch* b, cudaStream_t s) {
  msk_status st = bcuda(b, cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(unsigned int), s), "counter reset");
  for (size_t k = 0; k < b->items.size() && st == MSK_OK; ++k) {
    const msk_batch_item& it = b->items[k];
    if (it.paths == 0) continue;
    double* F = b->scratch + b->f_off[k];
    double* Wt = b->scratch + b->w_off[k];
    float* P = reinterpret_cast<float*>(b->scratch + b->p_off[k]);
    st = launch_brownian(it.ctx, it.steps, it.paths, F, false, s, true);   // float solves: float normals
    // the power norms are recomputed into the batch's own scratch on every run (a few
    // microseconds): the graph then depends on no state of the contexts' caches
    if (st == MSK_OK) st = launch_power_norms(it.ctx, it.order, it.steps, P, s);
    if (st == MSK_OK) st = launch_omega_tab(it.ctx, it.order, it.steps, it.paths, MSK_F32, F, Wt, P, s);
    // the megakernel takes each item's paths costliest first (the item table points at this order)
    long long* order_buf = reinterpret_cast<long long*>(b->scratch + b->o_off[k]);
    if (st == MSK_OK && b->variant != kPerGridVariant)
      st = launch_path_order(it.ctx, Wt, it.steps, it.paths, order_buf,
                             reinterpret_cast<unsigned long long*>(order_buf + it.paths), s);
    if (st != MSK_OK) b->err = it.ctx->err;
  }
  if (st != MSK_OK || b->n_units + b->n_tasks == 0) return st;
  if (b->variant == kPerGridVariant) {   // each item's own engine launch, one after another
    for (size_t k = 0; k < b->items.size() && st == MSK_OK; ++k) {
      const msk_batch_item& it = b->items[k];
      if (it.paths == 0) continue;
      long long* order_buf = reinterpret_cast<long long*>(b->scratch + b->o_off[k]);
      st = launch_magnus_queued(it.ctx, it.steps, it.paths, MSK_F32, b->scratch + b->w_off[k], it.u_out_dev,
                                it.status_dev, s, order_buf,
                                reinterpret_cast<unsigned long long*>(order_buf + it.paths));
      if (st != MSK_OK) b->err = it.ctx->err;
    }
    return st;
  }
  const BatchUnit* units = b->d_units;
  if (b->n_units > 0) {
    // interleaved units need the 512-thread megakernel; 256^2 units alone run on
    // 256-thread CTAs with the Taylor partial sum in registers
    const bool all_types = b->variant & 1;
    auto kern = all_types ? batch_kernel<kNT> : batch_kernel<kNT256>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(148 * 4, 1, 1);
    cfg.blockDim = dim3(all_types ? kNT : kNT256, 1, 1);
    cfg.dynamicSmemBytes = all_types ? batch_smem<kNT>() : batch_smem<kNT256>();
    cfg.stream = s;
    int nc = 0;
    st = bcuda(b, cudaOccupancyMaxActiveClusters(&nc, kern, &cfg), "occupancy clusters");
    if (st != MSK_OK) return st;
    if (nc < 1) return bfail(b, MSK_ERR_UNSUPPORTED, "batch cluster configuration cannot be scheduled");
    cfg.gridDim = dim3((unsigned)(std::min(nc, b->n_units) * 4), 1, 1);
    st = bcuda(b, cudaLaunchKernelEx(&cfg, kern, (const EngineArgs*)b->d_args, units, b->n_units, b->d_counter),
               "batch launch");
    if (st != MSK_OK) return st;
  }
  if (b->n_tasks > 0) {
    // a programmatic dependent of the megakernel: it may start once every
    // megakernel CTA is resident, on the SMs the clusters leave free, and takes
    // the rest as the megakernel's CTAs exit
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3((unsigned)std::min<int64_t>(b->items[0].ctx->num_sms, b->n_tasks), 1, 1);
    cfg.blockDim = dim3(kNT, 1, 1);
    cfg.dynamicSmemBytes = kTaskSmem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = b->n_units > 0 ? 1 : 0;
    st = bcuda(b, cudaLaunchKernelEx(&cfg, batch_task_kernel, (const EngineArgs*)b->d_args, units + b->n_units,
                                     b->n_tasks, b->d_counter),
               "batch task launch");
  }
  return st;
}

msk_status capture(msk_batch* b, cudaStream_t s) {
  drop_graph(b);
  msk_status st = bcuda(b, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (st != MSK_OK) return st;
  msk_status est = enqueue(b, s);
  cudaGraph_t g = nullptr;
  st = bcuda(b, cudaStreamEndCapture(s, &g), "end capture");
  if (est != MSK_OK) {
    if (g) cudaGraphDestroy(g);
    return est;
  }
  if (st != MSK_OK) return st;
  b->graph = g;
  return bcuda(b, cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
}

std::string batch_key(const msk_batch* b) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, b->device);
  std::string k = prop.name;
  for (const auto& it : b->items)
    k += "|" + std::to_string(it.ctx->d) + "x" + std::to_string(it.paths) + "o" + std::to_string(it.order) + "k" +
         std::to_string(it.steps);
  for (auto& ch : k)
    if (ch == ' ') ch = '_';
  return k;
}

int cached_variant(const char* path, const std::string& key) {
  if (!path || !*path) return -1;
  FILE* f = fopen(path, "r");
  if (!f) return -1;
  char line[4096];
  int v = -1;
  while (fgets(line, sizeof line, f)) {
    std::string l(line);
    const size_t sp = l.rfind(' ');
    if (sp != std::string::npos && l.substr(0, sp) == key) v = atoi(l.c_str() + sp + 1);
  }
  fclose(f);
  return v;
}

}  // namespace

extern "C" msk_status msk_batch_create(msk_batch** out, const msk_batch_item* items, int n_items,
                                       const char* tune_cache) {
  if (!out) return MSK_ERR_ARG;
  *out = nullptr;
  if (!items || n_items < 1) return MSK_ERR_ARG;
  const int dev = items[0].ctx ? items[0].ctx->device : -1;
  for (int k = 0; k < n_items; ++k) {
    const msk_batch_item& it = items[k];
    if (!it.ctx || it.ctx->device != dev) return MSK_ERR_ARG;
    const int d = it.ctx->d;
    if (d != 64 && d != 128 && d != 256) return MSK_ERR_UNSUPPORTED;
    if (it.ctx->xprof || it.ctx->gen) return MSK_ERR_UNSUPPORTED;   // batches run the constant-coefficient engine
    if (it.order < 1 || it.order > 3 || it.steps < 1 || it.ctx->n_fine % it.steps != 0 || it.paths < 0)
      return MSK_ERR_ARG;
    if (it.paths > 0 && !it.u_out_dev) return MSK_ERR_ARG;
  }
  msk_batch* b = new (std::nothrow) msk_batch();
  if (!b) return MSK_ERR_OOM;
  b->device = dev;
  b->items.assign(items, items + n_items);
  msk_status st = bcuda(b, cudaSetDevice(dev), "set device");
  size_t total = 0;
  for (int k = 0; k < n_items; ++k) {
    b->f_off.push_back(total);
    total += (size_t)items[k].paths * items[k].steps * MSK_NF;
    b->w_off.push_back(total);
    total += (size_t)items[k].paths * items[k].steps * MSK_NWT;
    b->o_off.push_back(total);
    total += (size_t)items[k].paths + 1;
    b->p_off.push_back(total);   // room for one row per step: the most any coefficient set needs
    total += ((size_t)items[k].steps * MSK_POW_J + 1) / 2;
  }
  if (st == MSK_OK) st = bcuda(b, cudaMalloc(&b->scratch, std::max<size_t>(total, 1) * sizeof(double)), "scratch");
  if (st == MSK_OK) st = bcuda(b, cudaMalloc(&b->d_counter, 2 * sizeof(unsigned int)), "counters");
  if (st == MSK_OK) st = bcuda(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "capture stream");
  if (st == MSK_OK) st = bcuda(b, cudaMalloc(&b->d_args, n_items * sizeof(EngineArgs)), "item table");
  for (int k = 0; k < n_items && st == MSK_OK; ++k) {
    const msk_batch_item& it = items[k];
    msk_ctx* c = it.ctx;
    EngineArgs a{};
    a.band = c->band;
    a.u0 = c->u0;
    a.Wt = b->scratch + b->w_off[k];
    a.dW = nullptr;
    a.out = it.u_out_dev;
    a.status = it.status_dev;
    a.work = c->work;
    a.paths = it.paths;
    a.steps = it.steps;
    a.dx = c->dx;
    a.T = c->T;
    a.s_cap = kMskScaleCap;
    a.tol32 = 0x1p-20f;   // float Taylor tolerance (see gen_theta.py)
    a.tol64 = 0x1p-53;
    a.c = coef_dev(c->coef);
    // the megakernel's path order (written on every run before the megakernel)
    a.order = reinterpret_cast<const long long*>(b->scratch + b->o_off[k]);
    b->args.push_back(a);
    st = msk_prepare_brownian(c, 0);
    if (st == MSK_OK) st = msk_prepare_omega(c);
    if (st != MSK_OK) b->err = c->err;
  }
  if (st == MSK_OK)
    st = bcuda(b, cudaMemcpy(b->d_args, b->args.data(), n_items * sizeof(EngineArgs), cudaMemcpyHostToDevice),
               "item table upload");
  if (st == MSK_OK)
    st = bcuda(b, cudaFuncSetAttribute(batch_kernel<kNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)batch_smem<kNT>()),
               "smem attribute");
  if (st == MSK_OK)
    st = bcuda(b, cudaFuncSetAttribute(batch_kernel<kNT256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)batch_smem<kNT256>()),
               "smem attribute");
  if (st == MSK_OK)
    st = bcuda(b, cudaFuncSetAttribute(batch_task_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTaskSmem),
               "smem attribute");
  if (st == MSK_OK) st = bcuda(b, cudaDeviceSynchronize(), "prepare");
  if (st == MSK_OK) {
    b->key = batch_key(b);
    const int v = cached_variant(tune_cache, b->key);
    st = set_variant(b, v >= 0 && v < kVariants ? v : 0);
  }
  if (st != MSK_OK) {
    msk_batch_destroy(b);
    return st;
  }
  *out = b;
  return MSK_OK;
}

extern "C" void msk_batch_destroy(msk_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  drop_graph(b);
  if (b->scratch) cudaFree(b->scratch);
  if (b->d_args) cudaFree(b->d_args);
  if (b->d_units) cudaFree(b->d_units);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

extern "C" const char* msk_batch_last_error(const msk_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" msk_status msk_batch_run(msk_batch* b, void* stream) {
  if (!b) return MSK_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  msk_status st = bcuda(b, cudaSetDevice(b->device), "set device");
  if (st != MSK_OK) return st;
  if (!b->exec) {
    // capture on the batch's own stream (capture is not possible on the legacy
    // default stream); the instantiated graph then runs on the caller's stream
    st = capture(b, b->cap_stream);
    if (st != MSK_OK) return st;
  }
  return bcuda(b, cudaGraphLaunch(b->exec, s), "graph launch");
}

extern "C" msk_status msk_batch_tune(msk_batch* b, void* stream, const char* tune_cache, int* variant_out,
                                     float* ms_out) {
  if (!b) return MSK_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  msk_status st = bcuda(b, cudaSetDevice(b->device), "set device");
  if (st != MSK_OK) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f, times[kVariants] = {0, 0, 0, 0, 0};
  int best_v = 0;
  for (int v = 0; v < kVariants && st == MSK_OK; ++v) {
    st = set_variant(b, v);
    if (st == MSK_OK) st = msk_batch_run(b, stream);            // capture + warm-up
    if (st != MSK_OK) break;
    cudaEventRecord(e0, s);
    st = msk_batch_run(b, stream);
    cudaEventRecord(e1, s);
    if (st == MSK_OK) st = bcuda(b, cudaEventSynchronize(e1), "tune sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    times[v] = ms;
    if (ms < best) {
      best = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MSK_OK) return st;
  st = set_variant(b, best_v);
  if (st != MSK_OK) return st;
  if (variant_out) *variant_out = best_v;
  if (ms_out)
    for (int v = 0; v < kVariants; ++v) ms_out[v] = times[v];
  if (tune_cache && *tune_cache) {
    FILE* f = fopen(tune_cache, "a");
    if (f) {
      fprintf(f, "%s %d\n", b->key.c_str(), best_v);
      fclose(f);
    }
  }
  return MSK_OK;
}

extern "C" int msk_batch_variant(const msk_batch* b) { return b ? b->variant : -1; }

extern "C" msk_status msk_batch_set_variant(msk_batch* b, int variant) {
  if (!b) return MSK_ERR_ARG;
  if (variant < 0 || variant >= kVariants) return bfail(b, MSK_ERR_ARG, "variant must be 0..4");
  msk_status st = bcuda(b, cudaSetDevice(b->device), "set device");
  if (st != MSK_OK) return st;
  return set_variant(b, variant);
}
