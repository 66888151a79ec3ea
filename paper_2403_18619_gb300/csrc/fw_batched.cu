// Batched solve: many independent graphs of different sizes in one persistent
// launch, replayed from a CUDA graph.
//
// Every graph keeps its own blocked-FW task queue (decode_task with its own R,
// block size and lookahead) and its own flags and snapshots.  The plan
// interleaves the graphs' queues into one global list in "stage waves": stage
// 0 of every graph, then stage 1 of every graph, ... (largest graphs first),
// each wave phase by phase (every graph's pivots, then remaining tiles, then
// panels, ...).  Each graph's tasks keep their relative order, so the global
// list is still a topological order of every graph's dependencies, and a
// graph's latency-bound pivot -> panel chain hides behind the other graphs'
// min-plus work.  One
// kernel (the warp-specialised engine with a runtime block size per task)
// drains the list.
//
// The block size of each graph comes from a per-size-class table, filled with
// defaults or measured by fw_autotune_bs on this GPU.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "fw_ws.cuh"

namespace fwk {

template <typename T>
struct BatchParams {
  const Args<T>* graphs;
  const int* bsv;
  const uint2* list;  // (graph, task index within the graph's queue)
  int64_t ntasks;
  unsigned* next;
  int* status;
  int* abort_flag;
  int64_t timeout_ns;
  uint64_t* trace;  // optional per-task trace (fw_options.trace of the plan)
  int trace_cap, trace_stride;
};

template <typename T>
struct BatchSrc {
  const Args<T>* graphs;
  const int* bsv;
  const uint2* list;
  int64_t ntasks;
  unsigned* next;
  int* status;
  int* abort_flag;
  int64_t timeout_ns;
  int skip_task = -1;
  uint64_t* trace = nullptr;
  int trace_cap = 0, trace_stride = 0;
  __device__ explicit BatchSrc(const BatchParams<T>& p)
      : graphs(p.graphs), bsv(p.bsv), list(p.list), ntasks(p.ntasks), next(p.next),
        status(p.status), abort_flag(p.abort_flag), timeout_ns(p.timeout_ns), trace(p.trace),
        trace_cap(p.trace_cap), trace_stride(p.trace_stride) {}
  __device__ int64_t total() const { return ntasks; }
  __device__ fwh::Task resolve(int64_t t, int& g) const {
    const uint2 e = list[t];
    g = (int)e.x;
    const Args<T>& a = graphs[g];
    return fwh::decode_task((int64_t)e.y, a.R, a.lookahead, a.stage_off);
  }
  __device__ const Args<T>& args(int g) const { return graphs[g]; }
  __device__ int bs(int g) const { return bsv[g]; }
};

template <typename T>
__global__ void __launch_bounds__(kWsThreads, 1) k_batched_ws(BatchParams<T> p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ WsBars wb;
  __shared__ CtaScratch cs;
  const BatchSrc<T> src(p);
  ws_engine<T, 0, 128>(src, smem, wb, cs);
}

// pred initialisation of every graph: blockIdx.y is the graph.
template <typename T>
__global__ void __launch_bounds__(256) k_batched_init(const Args<T>* graphs) {
  const Args<T> a = graphs[blockIdx.y];
  if (!a.P) return;  // distance-only
  const int64_t total = a.n * a.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / a.n, j = e - i * a.n;
    const T w = a.D[i * a.ld + j];
    a.P[i * a.ld + j] = (i != j && Num<T>::finite(w)) ? (int32_t)i : -1;
  }
}

// int32: every graph's via-coded predecessor entries become last hops (see
// ViaPred in fw_device.cuh); blockIdx.y is the graph.
__global__ void __launch_bounds__(256) k_batched_resolve(const Args<int32_t>* graphs) {
  const Args<int32_t> a = graphs[blockIdx.y];
  if (!a.P) return;  // distance-only
  const int64_t total = a.n * a.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / a.n, j = e - i * a.n;
    const int32_t pv = a.P[i * a.ld + j];
    if (pv <= -2) a.P[i * a.ld + j] = resolve_pred(pv, a.P, a.ld, j);
  }
}

}  // namespace fwk

namespace fwh {

// ----------------------------------------------------------- size classes ----

namespace {

constexpr int kClasses = 7;  // n <= 128, 256, 512, 1024, 2048, 4096, larger
const int64_t kClassMax[kClasses] = {128, 256, 512, 1024, 2048, 4096, 1 << 30};

// One table per element type (int32, fp32): the defaults are fw_autotune_bs's
// choices on GB300 (16 graphs per class); packed int32 keys favour BS = 128
// down to the smallest class, fp32's three-instruction relaxation BS = 32.
std::mutex g_table_mu;
int g_bs_table[2][kClasses] = {{128, 64, 64, 128, 128, 128, 128},
                               {32, 64, 64, 128, 128, 128, 128}};
int table_index(fw_dtype dt) { return dt == FW_F32 ? 1 : 0; }

int class_of(int64_t n) {
  for (int c = 0; c < kClasses; ++c)
    if (n <= kClassMax[c]) return c;
  return kClasses - 1;
}

int table_bs(int64_t n, fw_dtype dt) {
  std::lock_guard<std::mutex> lk(g_table_mu);
  return g_bs_table[table_index(dt)][class_of(n)];
}

constexpr size_t kAl = 256;
size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the debug shuffle's
// random stream.
uint64_t splitmix_next(uint64_t& x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// The global task list of `ns.size()` graphs with R[g] rounds each: (graph,
// task index in that graph's queue), in claim order; look[g] and offs[g]
// receive each graph's lookahead and queue stage offsets.  Stage waves, phase by phase: a graph's stage s is
// [pivot(s)] [its first remaining tiles of round s-1] [panels(s)] [the rest
// of round s-1] [round s's tiles in tile row / column s+1] (decode_task's
// layout), and the wave emits segment 0 of every graph, then segment 1 of
// every graph, ...  So the tiles between one graph's pivot and its panels
// are every graph's (a pivot takes about as long as 3 remaining tiles, far
// more than its own graph's tiles cover when many graphs share the GPU), and
// each graph's own tasks keep their order: the list stays a topological
// order of every graph's dependencies.
//
// shuffle != 0 permutes each wave segment (Fisher-Yates, seeded): a segment
// holds one phase of one round of each graph -- pivots, remaining tiles of
// one round, or panels of one round -- and no task of a segment depends on
// another of the same segment, so every permutation is still a topological
// order (a stress of the dependency protocol under other claim orders).
fw_status build_task_list(const std::vector<int64_t>& ns, const std::vector<int>& R, int sms,
                          uint64_t shuffle, std::vector<uint2>& list, std::vector<int64_t>& look,
                          std::vector<std::vector<unsigned>>& offs) {
  const int64_t B = (int64_t)ns.size();
  std::vector<int64_t> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return ns[x] > ns[y]; });
  offs.assign(B, {});
  int maxR = 0;
  int64_t total = 0;
  look.assign(B, 0);
  for (int64_t g = 0; g < B; ++g) {
    look[g] = auto_lookahead(R[g], sms);
    offs[g].resize(R[g] + 2);
    fill_stage_offsets(R[g], look[g], offs[g].data());
    maxR = std::max(maxR, R[g]);
    total += (int64_t)R[g] * R[g] * R[g];
  }
  if (total >= (int64_t)1 << 31) return FW_ERR_UNSUPPORTED;
  list.clear();
  list.reserve(total);
  uint64_t rng = shuffle;
  for (int s = 0; s <= maxR; ++s)
    for (int seg = 0; seg < 5; ++seg) {
      const size_t wave0 = list.size();
      for (int64_t oi = 0; oi < B; ++oi) {
        const int64_t g = order[oi];
        const int Rg = R[g];
        if (s > Rg) continue;
        const int64_t np = s < Rg ? 2 * (int64_t)(Rg - 1) : 0;
        const int64_t nrest = s >= 1 ? size_rest(Rg, s - 1) : 0;
        const int64_t gl =
            s >= 1 && s < Rg ? std::min<int64_t>(look[g], nrest) : (s == Rg ? nrest : 0);
        const int64_t len[5] = {s < Rg ? 1 : 0, gl, np, s >= 1 && s < Rg ? nrest - gl : 0,
                                s < Rg ? size_L(Rg, s) : 0};
        int64_t first = offs[g][s];
        for (int k = 0; k < seg; ++k) first += len[k];
        for (int64_t t = first; t < first + len[seg]; ++t)
          list.push_back(make_uint2((unsigned)g, (unsigned)t));
      }
      if (shuffle)
        for (size_t k = list.size() - wave0; k > 1; --k)
          std::swap(list[wave0 + k - 1], list[wave0 + splitmix_next(rng) % k]);
    }
  if ((int64_t)list.size() != total) return FW_ERR_CUDA;  // the segments cover every stage
  return FW_OK;
}

}  // namespace

}  // namespace fwh

// ------------------------------------------------------------------ plan ----

struct fw_batched_plan {
  int device = 0;
  fw_dtype dtype = FW_I32;
  fw_options opt{};
  int64_t batch = 0;
  std::vector<int64_t> n, ld;
  std::vector<int> bs, R;
  void* dmem = nullptr;  // every device table and workspace of the plan
  size_t dbytes = 0;
  void* d_args = nullptr;
  int* d_bs = nullptr;
  uint2* d_list = nullptr;
  int64_t ntasks = 0;
  unsigned* d_next = nullptr;  // claim counter
  int* d_abort = nullptr;
  size_t flags_bytes = 0;      // the contiguous region zeroed before each solve
  void* d_flags = nullptr;
  std::vector<unsigned char> h_args;  // host copy of the per-graph Args
  size_t args_size = 0;
  std::vector<void*> cur_dist, cur_pred;
  int* cur_status = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int grid = 0;
  std::mutex mu;
};

namespace fwh {

int* status_word_for(cudaStream_t s);  // fw_api.cu

namespace {

template <typename T>
fw_status plan_build(fw_batched_plan* p) {
  using A = fwk::Args<T>;
  const int64_t B = p->batch;
  p->args_size = sizeof(A);
  // per-graph workspace sizes
  std::vector<size_t> ws_bytes(B), flag_off(B), ws_off(B);
  size_t flags = 0;
  for (int64_t g = 0; g < B; ++g) {
    flag_off[g] = flags;
    flags += al(((size_t)p->R[g] * p->R[g] + 2 * (size_t)p->R[g]) * 4 + 4 * 4);  // ver+done+ctr
  }
  flags += al(4 * 4);  // next counter + abort
  p->flags_bytes = flags;
  size_t off = al(flags);
  // per-graph stage offsets + snapshots (solve_ws_bytes covers flags too; the
  // flag part of that carve is simply unused)
  for (int64_t g = 0; g < B; ++g) {
    ws_off[g] = off;
    ws_bytes[g] = solve_ws_bytes(p->R[g], p->bs[g]);
    off += al(ws_bytes[g]);
  }
  // the global task list (stage waves, largest graphs first)
  std::vector<uint2> list;
  std::vector<int64_t> look;
  std::vector<std::vector<unsigned>> offs;
  const fw_status lst =
      build_task_list(p->n, p->R, num_sms(), p->opt.debug_shuffle, list, look, offs);
  if (lst != FW_OK) return lst;
  p->ntasks = (int64_t)list.size();
  const size_t list_off = off;
  off += al(list.size() * sizeof(uint2));
  const size_t args_off = off;
  off += al((size_t)B * sizeof(A));
  const size_t bs_off = off;
  off += al((size_t)B * 4);
  p->dbytes = off + kAl;
  if (cudaMalloc(&p->dmem, p->dbytes) != cudaSuccess) {
    cudaGetLastError();
    p->dmem = nullptr;
    return FW_ERR_NOMEM;
  }
  char* base = reinterpret_cast<char*>(p->dmem);
  p->d_flags = base;
  p->d_next = reinterpret_cast<unsigned*>(base + flags - al(4 * 4));
  p->d_abort = reinterpret_cast<int*>(p->d_next + 1);
  p->d_list = reinterpret_cast<uint2*>(base + list_off);
  p->d_args = base + args_off;
  p->d_bs = reinterpret_cast<int*>(base + bs_off);

  // host copies of every graph's Args (D / P / status patched at solve time)
  p->h_args.assign((size_t)B * sizeof(A), 0);
  A* ha = reinterpret_cast<A*>(p->h_args.data());
  std::vector<unsigned> all_offs;
  for (int64_t g = 0; g < B; ++g) {
    SolveWs w = carve_solve_ws(base + ws_off[g], p->R[g], p->bs[g]);
    A a{};
    a.D = nullptr;
    a.P = nullptr;
    a.n = p->n[g];
    a.ld = p->ld[g];
    a.R = p->R[g];
    a.slot_tiles = w.slot_tiles;
    a.ver = reinterpret_cast<int*>(base + flag_off[g]);
    a.done = a.ver + (size_t)p->R[g] * p->R[g];
    a.ctr = reinterpret_cast<unsigned*>(a.done + 2 * (size_t)p->R[g]);
    a.abort_flag = p->d_abort;
    a.status = nullptr;
    a.stage_off = w.stage_off;
    a.lookahead = (int)look[g];
    a.skip_task = -1;
    a.timeout_ns = p->opt.timeout_ns > 0 ? p->opt.timeout_ns : 2000000000LL;
    a.packed = p->opt.packed_keys ? 1 : 0;
    a.piv = reinterpret_cast<T*>(w.piv);
    a.pivP = w.pivP;
    a.colK = w.colK;
    a.colR = reinterpret_cast<T*>(w.colR);
    a.colB = w.colB;
    a.rowK = w.rowK;
    a.rowR = reinterpret_cast<T*>(w.rowR);
    a.rowP = w.rowP;
    a.rowB = w.rowB;
    a.trace = nullptr;
    ha[g] = a;
    if (cudaMemcpy(w.stage_off, offs[g].data(), offs[g].size() * 4, cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return FW_ERR_CUDA;
  }
  if (cudaMemcpy(p->d_list, list.data(), list.size() * sizeof(uint2), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(p->d_bs, p->bs.data(), (size_t)B * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return FW_ERR_CUDA;

  const size_t smem = fwk::WsLayout<128, T>::bytes();
  auto kern = fwk::k_batched_ws<T>;
  const int occ = kernel_setup(reinterpret_cast<const void*>(kern), smem, fwk::kWsThreads);
  if (occ < 1) return FW_ERR_CUDA;
  int64_t grid = (int64_t)occ * num_sms();
  if (p->opt.grid > 0 && p->opt.grid < grid) grid = p->opt.grid;
  if (grid > p->ntasks) grid = p->ntasks;
  p->grid = (int)std::max<int64_t>(grid, 1);
  return FW_OK;
}

// Enqueue (or capture) the work of one batched solve on stream s.
template <typename T>
cudaError_t enqueue(fw_batched_plan* p, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(p->d_flags, 0, p->flags_bytes, s)) != cudaSuccess) return e;
  int64_t maxn2 = 0;
  for (int64_t g = 0; g < p->batch; ++g) maxn2 = std::max(maxn2, p->n[g] * p->n[g]);
  const unsigned gx = (unsigned)std::min<int64_t>((maxn2 + 255) / 256, 64);
  const auto* args = reinterpret_cast<const fwk::Args<T>*>(p->d_args);
  for (int64_t g0 = 0; g0 < p->batch; g0 += 65535) {
    const unsigned gy = (unsigned)std::min<int64_t>(p->batch - g0, 65535);
    fwk::k_batched_init<T><<<dim3(gx, gy), 256, 0, s>>>(args + g0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  fwk::BatchParams<T> bp;
  bp.graphs = args;
  bp.bsv = p->d_bs;
  bp.list = p->d_list;
  bp.ntasks = p->ntasks;
  bp.next = p->d_next;
  bp.status = p->cur_status;
  bp.abort_flag = p->d_abort;
  bp.timeout_ns = p->opt.timeout_ns > 0 ? p->opt.timeout_ns : 2000000000LL;
  bp.trace = p->opt.trace;
  bp.trace_cap = (int)p->opt.trace_cap;
  bp.trace_stride = p->opt.trace_stride;
  cudaLaunchConfig_t lc{};
  lc.gridDim = dim3((unsigned)p->grid);
  lc.blockDim = dim3(fwk::kWsThreads);
  lc.dynamicSmemBytes = fwk::WsLayout<128, T>::bytes();
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  if ((e = cudaLaunchKernelEx(&lc, fwk::k_batched_ws<T>, bp)) != cudaSuccess) return e;
  if constexpr (fwk::ViaPred<T>::kOn) {
    for (int64_t g0 = 0; g0 < p->batch; g0 += 65535) {
      const unsigned gy = (unsigned)std::min<int64_t>(p->batch - g0, 65535);
      fwk::k_batched_resolve<<<dim3(gx, gy), 256, 0, s>>>(
          reinterpret_cast<const fwk::Args<int32_t>*>(args + g0));
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <typename T>
fw_status solve_plan(fw_batched_plan* p, void* const* dist, int32_t* const* pred,
                     cudaStream_t s) {
  using A = fwk::Args<T>;
  int* st = status_word_for(s);
  if (!st) return FW_ERR_NOMEM;
  bool changed = st != p->cur_status;
  for (int64_t g = 0; g < p->batch && !changed; ++g)
    changed = dist[g] != p->cur_dist[g] || (void*)(pred ? pred[g] : nullptr) != p->cur_pred[g];
  if (changed) {
    // New buffers: refresh the device table of per-graph arguments, which the
    // recorded kernels read when they run, with a copy ordered on s behind
    // the previous solve (the caller keeps a plan's solves from overlapping:
    // one stream, or the previous solve finished before another stream
    // takes the plan).  Only a new status word (a solve on another stream)
    // changes a kernel parameter of the recorded graph and needs a new
    // recording, after that stream's earlier work.
    const bool restream = st != p->cur_status;
    if (restream && p->cur_status && cudaStreamSynchronize(s) != cudaSuccess) return FW_ERR_CUDA;
    A* ha = reinterpret_cast<A*>(p->h_args.data());
    for (int64_t g = 0; g < p->batch; ++g) {
      ha[g].D = reinterpret_cast<T*>(dist[g]);
      ha[g].P = pred ? pred[g] : nullptr;
      ha[g].status = st;
      p->cur_dist[g] = dist[g];
      p->cur_pred[g] = ha[g].P;
    }
    p->cur_status = st;
    if (cudaMemcpyAsync(p->d_args, p->h_args.data(), p->h_args.size(), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
      return FW_ERR_CUDA;
    if (restream) {
      if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
      }
      if (p->graph) {
        cudaGraphDestroy(p->graph);
        p->graph = nullptr;
      }
    }
  }
  if (!p->exec) {
    if (!p->cap_stream &&
        cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return FW_ERR_CUDA;
    if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return FW_ERR_CUDA;
    const cudaError_t e = enqueue<T>(p, p->cap_stream);
    cudaGraph_t gr = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess || !gr) {
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      return FW_ERR_CUDA;
    }
    p->graph = gr;
    if (cudaGraphInstantiate(&p->exec, gr, 0) != cudaSuccess) {
      cudaGetLastError();
      p->exec = nullptr;
      return FW_ERR_CUDA;
    }
  }
  if (p->opt.ev_start) cudaEventRecord(reinterpret_cast<cudaEvent_t>(p->opt.ev_start), s);
  if (cudaGraphLaunch(p->exec, s) != cudaSuccess) return FW_ERR_CUDA;
  if (p->opt.ev_stop) cudaEventRecord(reinterpret_cast<cudaEvent_t>(p->opt.ev_stop), s);
  return FW_OK;
}

void plan_free(fw_batched_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->dmem) cudaFree(p->dmem);
  p->exec = nullptr;
  p->graph = nullptr;
  p->cap_stream = nullptr;
  p->dmem = nullptr;
}

// ------------------------------------------------------------- autotuning ----

// Timing workload of the autotuner (any valid graph will do): a dense digraph
// with int32 weights in [1, 100] (or fp32 in (0, 1]) from a hash of (g, i, j).
template <typename T>
__global__ void k_tune_fill(T* D, int64_t n, int64_t ld, int g) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    uint32_t h = (uint32_t)(i * 73856093u) ^ (uint32_t)(j * 19349663u) ^ (uint32_t)(g * 83492791u);
    h ^= h >> 13;
    h *= 0x5bd1e995u;
    h ^= h >> 15;
    T v;
    if (i == j) v = T(0);
    else if ((h & 7u) < 3u) v = fwk::Num<T>::inf();  // ~37% missing edges
    else if constexpr (fwk::Num<T>::kInt) v = (T)(1 + (h >> 8) % 100);
    else v = (T)(((h >> 8) & 0xffffu) + 1) * (1.0f / 65536.0f);
    D[i * ld + j] = v;
  }
}

}  // namespace
}  // namespace fwh

using namespace fwh;

extern "C" {

fw_status fw_batched_plan_create(fw_batched_plan** plan, const int64_t* n, const int64_t* ld,
                                 int64_t batch, fw_dtype dtype, const fw_options* opt) {
  if (!plan) return FW_ERR_ARG;
  *plan = nullptr;
  if (!n || !ld || batch < 1 || batch > 65536) return FW_ERR_ARG;
  if (dtype == FW_I64 || dtype == FW_F64) return FW_ERR_UNSUPPORTED;  // 32-bit types only
  if (dtype != FW_I32 && dtype != FW_F32) return FW_ERR_ARG;
  fw_options o;
  fw_options_default(&o);
  if (opt) o = *opt;
  if (o.bs != 0 && o.bs != 32 && o.bs != 64 && o.bs != 128) return FW_ERR_ARG;
  if (o.trace && (o.trace_cap <= 0 || o.trace_cap > (1 << 30) || o.trace_stride <= 0))
    return FW_ERR_ARG;
  for (int64_t g = 0; g < batch; ++g)
    if (n[g] < 1 || n[g] > 131072 || ld[g] < n[g] || (ld[g] % 4) != 0) return FW_ERR_ARG;
  auto* p = new fw_batched_plan();
  cudaGetDevice(&p->device);
  p->dtype = dtype;
  p->opt = o;
  p->batch = batch;
  p->n.assign(n, n + batch);
  p->ld.assign(ld, ld + batch);
  p->bs.resize(batch);
  p->R.resize(batch);
  for (int64_t g = 0; g < batch; ++g) {
    p->bs[g] = o.bs ? o.bs : table_bs(n[g], dtype);
    p->R[g] = (int)((n[g] + p->bs[g] - 1) / p->bs[g]);
    if (p->R[g] > 1024) {
      delete p;
      return FW_ERR_UNSUPPORTED;
    }
  }
  p->cur_dist.assign(batch, nullptr);
  p->cur_pred.assign(batch, nullptr);
  const fw_status st = dtype == FW_I32 ? plan_build<int32_t>(p) : plan_build<float>(p);
  if (st != FW_OK) {
    plan_free(p);
    delete p;
    return st;
  }
  *plan = p;
  return FW_OK;
}

fw_status fw_batched_task_list(const int64_t* n, const int32_t* bs, int64_t batch, int32_t sms,
                               const fw_options* opt, int32_t* out, int64_t cap, int64_t* count) {
  if (!n || !bs || !out || !count || batch < 1 || batch > 65536 || sms < 1 || cap < 0)
    return FW_ERR_ARG;
  fw_options o;
  fw_options_default(&o);
  if (opt) o = *opt;
  std::vector<int64_t> ns(n, n + batch);
  std::vector<int> R(batch);
  for (int64_t g = 0; g < batch; ++g) {
    if (ns[g] < 1 || ns[g] > 131072 || (bs[g] != 32 && bs[g] != 64 && bs[g] != 128))
      return FW_ERR_ARG;
    const int64_t r = (ns[g] + bs[g] - 1) / bs[g];
    if (r > 1024) return FW_ERR_UNSUPPORTED;
    R[g] = (int)r;
  }
  std::vector<uint2> list;
  std::vector<int64_t> look;
  std::vector<std::vector<unsigned>> offs;
  const fw_status st = build_task_list(ns, R, sms, o.debug_shuffle, list, look, offs);
  if (st != FW_OK) return st;
  *count = (int64_t)list.size();
  if (cap < *count) return FW_ERR_ARG;
  for (size_t k = 0; k < list.size(); ++k) {
    out[2 * k] = (int32_t)list[k].x;
    out[2 * k + 1] = (int32_t)list[k].y;
  }
  return FW_OK;
}

fw_status fw_solve_batched(fw_batched_plan* p, void* const* dist, int32_t* const* pred,
                           void* stream) {
  if (!p || !dist) return FW_ERR_ARG;  // pred null: distance-only for every graph
  for (int64_t g = 0; g < p->batch; ++g) {
    int32_t* pg = pred ? pred[g] : nullptr;
    if (!dist[g] || dist[g] == (void*)pg) return FW_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(dist[g]) & 15) || (reinterpret_cast<uintptr_t>(pg) & 15))
      return FW_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return FW_ERR_ARG;
  std::lock_guard<std::mutex> lk(p->mu);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  return p->dtype == FW_I32 ? solve_plan<int32_t>(p, dist, pred, s)
                            : solve_plan<float>(p, dist, pred, s);
}

fw_status fw_batched_plan_info(const fw_batched_plan* p, int32_t* bs_per_graph,
                               int64_t* total_tasks) {
  if (!p) return FW_ERR_ARG;
  if (bs_per_graph)
    for (int64_t g = 0; g < p->batch; ++g) bs_per_graph[g] = p->bs[g];
  if (total_tasks) *total_tasks = p->ntasks;
  return FW_OK;
}

fw_status fw_batched_plan_destroy(fw_batched_plan* p) {
  if (!p) return FW_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != p->device) cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  plan_free(p);
  if (dev != p->device) cudaSetDevice(dev);
  delete p;
  return FW_OK;
}

fw_status fw_bs_table(fw_dtype dtype, int32_t* table, int32_t set) {
  if (!table) return FW_ERR_ARG;
  if (dtype == FW_I64 || dtype == FW_F64) return FW_ERR_UNSUPPORTED;  // no batched path
  if (dtype != FW_I32 && dtype != FW_F32) return FW_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_table_mu);
  int* t = g_bs_table[table_index(dtype)];
  if (set) {
    for (int c = 0; c < kClasses; ++c)
      if (table[c] != 32 && table[c] != 64 && table[c] != 128) return FW_ERR_ARG;
    for (int c = 0; c < kClasses; ++c) t[c] = table[c];
  } else {
    for (int c = 0; c < kClasses; ++c) table[c] = t[c];
  }
  return FW_OK;
}

fw_status fw_autotune_bs(fw_dtype dtype, int64_t graphs_per_class, int64_t max_n, void* stream,
                         int32_t* table_out, double* ms_out) {
  if (dtype == FW_I64 || dtype == FW_F64) return FW_ERR_UNSUPPORTED;  // 32-bit types only
  if (dtype != FW_I32 && dtype != FW_F32) return FW_ERR_ARG;
  if (graphs_per_class < 1 || graphs_per_class > 4096 || max_n < 1) return FW_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int32_t table[kClasses];
  fw_bs_table(dtype, table, 0);
  const int cand[3] = {32, 64, 128};
  for (int c = 0; c < kClasses; ++c) {
    const int64_t n = std::min<int64_t>(c + 1 < kClasses ? kClassMax[c] : 8192, max_n);
    if (c > 0 && n <= kClassMax[c - 1]) break;  // classes above max_n keep their entry
    const int64_t ld = (n + 3) / 4 * 4;
    const size_t bytes = (size_t)n * ld * 4;
    std::vector<void*> dd(graphs_per_class), pp(graphs_per_class);
    void* buf = nullptr;
    if (cudaMalloc(&buf, bytes * 2 * graphs_per_class) != cudaSuccess) {
      cudaGetLastError();
      return FW_ERR_NOMEM;
    }
    std::vector<int64_t> ns(graphs_per_class, n), lds(graphs_per_class, ld);
    for (int64_t g = 0; g < graphs_per_class; ++g) {
      dd[g] = (char*)buf + 2 * g * bytes;
      pp[g] = (char*)buf + (2 * g + 1) * bytes;
    }
    double best_ms = 1e30;
    int best = table[c];
    for (int bi = 0; bi < 3; ++bi) {
      fw_options o;
      fw_options_default(&o);
      o.bs = cand[bi];
      fw_batched_plan* plan = nullptr;
      if (fw_batched_plan_create(&plan, ns.data(), lds.data(), graphs_per_class, dtype, &o) !=
          FW_OK)
        continue;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float total = 0;
      bool ok = true;
      for (int rep = 0; rep < 3 && ok; ++rep) {
        for (int64_t g = 0; g < graphs_per_class; ++g) {
          if (dtype == FW_I32)
            k_tune_fill<int32_t><<<64, 256, 0, s>>>((int32_t*)dd[g], n, ld, (int)g);
          else
            k_tune_fill<float><<<64, 256, 0, s>>>((float*)dd[g], n, ld, (int)g);
        }
        cudaEventRecord(e0, s);
        ok = fw_solve_batched(plan, dd.data(), (int32_t* const*)pp.data(), stream) == FW_OK;
        cudaEventRecord(e1, s);
        ok = ok && fw_sync_status(stream) == FW_OK;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) total += ms;  // the first run records the graph
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      fw_batched_plan_destroy(plan);
      if (ok && total / 2 < best_ms) {
        best_ms = total / 2;
        best = cand[bi];
      }
    }
    cudaFree(buf);
    table[c] = best;
    if (ms_out) ms_out[c] = best_ms;
  }
  fw_bs_table(dtype, table, 1);
  if (table_out)
    for (int c = 0; c < kClasses; ++c) table_out[c] = table[c];
  return FW_OK;
}

}  // extern "C"
