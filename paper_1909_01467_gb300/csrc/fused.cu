// Fused applications over many problems (the batched form): one launch per dependency level
// runs the solves of every problem at that level (the union of the problems' own levels),
// one kernel resets all problems' traces and one sums all problems' lanes; the whole
// application is captured once as a CUDA graph and replayed.  The problems' inputs and
// outputs change from application to application (the FGMRES basis vectors), so the graph
// reads them from a device table that is refreshed before each replay, with a flag that
// leaves out the problems that are not applied (converged solves): their CTAs exit at once.
// Requires problems with the same sweep-front geometry (line width, padded width, lines)
// and the same kernel form (two CTAs per solve on twisted factors, or one CTA per solve),
// complex64.  lsweep_solve_batch_fused runs the problems' FGMRES processes in lockstep on
// top of it.
#include <algorithm>
#include <vector>

#include "front.cuh"

namespace lsw {

cudaError_t launch_front_fused(Ctx& c, const Task* tasks, int off, int count,
                               const FrontArgs* table, cudaStream_t stream);

// per problem: traces to reset, lanes to sum into z
struct FusedVec {
  float2* trace;
  long long trace_elems;
  const float2* lane;
  double2* z;
  long long Next;
  int skip;
  int pad;
};

__global__ void k_fused_reset(const FusedVec* __restrict__ v) {
  const FusedVec f = v[blockIdx.y];
  if (f.skip) return;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < f.trace_elems;
       t += (long long)gridDim.x * blockDim.x)
    f.trace[t] = make_float2(0.f, 0.f);
}

// z = the sum of the lanes, in the order of k_sum_lanes (lane 0 + lane 1 + ... in FP64)
__global__ void k_fused_sum(const FusedVec* __restrict__ v) {
  const FusedVec f = v[blockIdx.y];
  if (f.skip) return;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < f.Next;
       t += (long long)gridDim.x * blockDim.x) {
    double2 s = widen(f.lane[t]);
    s = s + widen(f.lane[f.Next + t]);
#pragma unroll
    for (int l = 2; l < kLanes; ++l) s = s + widen(f.lane[(size_t)l * f.Next + t]);
    f.z[t] = s;
  }
}

struct Fused {
  std::vector<Ctx*> cs;
  Task* d_tasks = nullptr;
  FrontArgs* d_args = nullptr;
  FusedVec* d_vec = nullptr;
  FrontArgs* h_args = nullptr;     // pinned mirrors, refreshed before each replay
  FusedVec* h_vec = nullptr;
  std::vector<Launch> levels;
  long long max_next = 0, max_trace = 0;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t a0 = nullptr, a1 = nullptr;
  std::vector<cudaEvent_t> ready;  // per problem: its stream's work before an application

  ~Fused() {
    if (stream) cudaStreamSynchronize(stream);
    for (cudaEvent_t e : ready)
      if (e) cudaEventDestroy(e);
    if (exec) cudaGraphExecDestroy(exec);
    if (a0) cudaEventDestroy(a0);
    if (a1) cudaEventDestroy(a1);
    if (stream) cudaStreamDestroy(stream);
    for (void* p : {(void*)d_tasks, (void*)d_args, (void*)d_vec})
      if (p) cs[0]->mem.put(p);
    if (h_args) cudaFreeHost(h_args);
    if (h_vec) cudaFreeHost(h_vec);
    cudaGetLastError();
  }

  // the captured application: trace reset, every fused level, lane sums
  cudaError_t launches() {
    const unsigned np = (unsigned)cs.size();
    const unsigned gr = (unsigned)std::min<long long>(64, (max_trace + 255) / 256);
    k_fused_reset<<<dim3(std::max(1u, gr), np), 256, 0, stream>>>(d_vec);
    cudaError_t e = cudaGetLastError();
    for (size_t l = 0; e == cudaSuccess && l < levels.size(); ++l)
      e = launch_front_fused(*cs[0], d_tasks, levels[l].off, levels[l].count, d_args, stream);
    if (e != cudaSuccess) return e;
    const unsigned gs = (unsigned)std::min<long long>(256, (max_next + 255) / 256);
    k_fused_sum<<<dim3(std::max(1u, gs), np), 256, 0, stream>>>(d_vec);
    return cudaGetLastError();
  }

  int build(const std::vector<Ctx*>& handles, std::string& msg) {
    cs = handles;
    const Ctx& r0 = *cs[0];
    for (Ctx* c : cs) {
      if (!c->c64() || c->p.windows || c->cube || c->dim != r0.dim || c->bmax != r0.bmax ||
          c->bpmax != r0.bpmax || c->Lmax != r0.Lmax || front_form(*c) != front_form(r0) ||
          front_form(r0) == 0) {
        msg = "problems need complex64 factors, no windows, no cube CDD, the same line width, "
              "padded width "
              "and line count, and the same sweep-front form (two CTAs per solve on twisted "
              "factors, or one CTA per solve)";
        return LSWEEP_EINVAL;
      }
    }
    // the union of the problems' dependency levels, level by level
    std::vector<Task> tasks;
    size_t nlev = 0;
    for (Ctx* c : cs) nlev = std::max(nlev, c->launches.size());
    for (size_t l = 0; l < nlev; ++l) {
      const int off = (int)tasks.size();
      for (size_t p = 0; p < cs.size(); ++p) {
        const Ctx* c = cs[p];
        if (l >= c->launches.size()) continue;
        const Launch& L = c->launches[l];
        for (int t = 0; t < L.count; ++t) {
          Task x = c->tasks[L.off + t];
          x.kind = x.kind | (int)(p << 8);
          tasks.push_back(x);
        }
      }
      if ((int)tasks.size() > off) levels.push_back({off, (int)tasks.size() - off});
    }
    const size_t np = cs.size();
    auto ok = [&](cudaError_t e) {
      if (e == cudaSuccess) return true;
      cudaGetLastError();
      msg = std::string("fused application: ") + cudaGetErrorString(e);
      return false;
    };
    d_tasks = static_cast<Task*>(cs[0]->mem.get(std::max<size_t>(16, tasks.size() * sizeof(Task))));
    d_args = static_cast<FrontArgs*>(cs[0]->mem.get(np * sizeof(FrontArgs)));
    d_vec = static_cast<FusedVec*>(cs[0]->mem.get(np * sizeof(FusedVec)));
    if (!d_tasks || !d_args || !d_vec) {
      cudaGetLastError();
      msg = "fused application: device allocation failed";
      return LSWEEP_ENOMEM;
    }
    if (!ok(cudaMallocHost(&h_args, np * sizeof(FrontArgs))) ||
        !ok(cudaMallocHost(&h_vec, np * sizeof(FusedVec))) ||
        !ok(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking)) ||
        !ok(cudaEventCreate(&a0)) || !ok(cudaEventCreate(&a1)))
      return LSWEEP_ENOMEM;
    ready.assign(np, nullptr);
    for (size_t p = 0; p < np; ++p)
      if (!ok(cudaEventCreateWithFlags(&ready[p], cudaEventDisableTiming))) return LSWEEP_ENOMEM;
    for (size_t p = 0; p < np; ++p) {
      const Ctx& c = *cs[p];
      FrontArgs a{};
      a.subs = c.d_subs;
      a.lcoef = c.d_lcoef;
      a.cstride = c.node_elems;
      a.fac = c.d_fac;
      a.lane = c.d_lane;
      a.Next = c.Next;
      a.trace = c.d_trace;
      a.W = c.trace_W;
      a.nsub = (int)c.subs.size();
      a.q = c.q;
      a.r = c.r;
      a.pz = c.pz;
      a.dim = c.dim;
      a.Ne = c.Ne;
      a.spin = c.spin();
      a.skip = 1;
      h_args[p] = a;
      FusedVec v{};
      v.trace = reinterpret_cast<float2*>(c.d_trace);
      v.trace_elems = (long long)c.n_trace_arr * c.subs.size() * 2 * c.trace_W;
      v.lane = reinterpret_cast<const float2*>(c.d_lane);
      v.Next = c.Next;
      v.skip = 1;
      h_vec[p] = v;
      max_next = std::max(max_next, c.Next);
      max_trace = std::max(max_trace, v.trace_elems);
    }
    if (!ok(cudaMemcpyAsync(d_tasks, tasks.data(), tasks.size() * sizeof(Task),
                            cudaMemcpyHostToDevice, stream)) ||
        !ok(cudaMemcpyAsync(d_args, h_args, np * sizeof(FrontArgs), cudaMemcpyHostToDevice, stream)) ||
        !ok(cudaMemcpyAsync(d_vec, h_vec, np * sizeof(FusedVec), cudaMemcpyHostToDevice, stream)) ||
        !ok(cudaStreamSynchronize(stream)))
      return LSWEEP_ECUDA;
    // one eager run with every problem left out sets the kernels' attributes; then capture
    if (!ok(launches()) || !ok(cudaStreamSynchronize(stream))) return LSWEEP_ECUDA;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = launches();
      cudaError_t e2 = cudaStreamEndCapture(stream, &graph);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (!ok(e)) return LSWEEP_ECUDA;
    return LSWEEP_OK;
  }

  // z[p] = A~^-1 r[p] for the problems with active[p]; completes a1 on `stream`
  int apply(const std::vector<char>& active, const std::vector<const double2*>& r,
            const std::vector<double2*>& z, std::string& msg) {
    const size_t np = cs.size();
    for (size_t p = 0; p < np; ++p) {
      h_args[p].rin = active[p] ? r[p] : nullptr;
      h_args[p].skip = active[p] ? 0 : 1;
      h_vec[p].z = active[p] ? z[p] : nullptr;
      h_vec[p].skip = active[p] ? 0 : 1;
    }
    // the inputs are written on the problems' own streams: wait for that work
    cudaError_t e = cudaSuccess;
    for (size_t p = 0; p < np && e == cudaSuccess; ++p) {
      if (!active[p]) continue;
      e = cudaEventRecord(ready[p], cs[p]->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ready[p], 0);
    }
    if (e == cudaSuccess) e = cudaEventRecord(a0, stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_args, h_args, np * sizeof(FrontArgs), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_vec, h_vec, np * sizeof(FusedVec), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, stream);
    if (e == cudaSuccess) e = cudaEventRecord(a1, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      msg = std::string("fused application: ") + cudaGetErrorString(e);
      return LSWEEP_ECUDA;
    }
    cs[0]->kernels += (long long)levels.size() + 2;
    return LSWEEP_OK;
  }
};

Fused* make_fused(const std::vector<Ctx*>& cs, int& rc, std::string& msg) {
  Fused* f = new (std::nothrow) Fused();
  if (!f) {
    rc = LSWEEP_ENOMEM;
    msg = "host allocation failed";
    return nullptr;
  }
  rc = f->build(cs, msg);
  if (rc) {
    delete f;
    return nullptr;
  }
  return f;
}

int fused_apply(Fused* f, const std::vector<char>& active, const std::vector<const double2*>& r,
                const std::vector<double2*>& z, std::string& msg) {
  return f->apply(active, r, z, msg);
}

cudaEvent_t fused_done(Fused* f) { return f->a1; }
cudaEvent_t fused_start(Fused* f) { return f->a0; }
size_t fused_levels(Fused* f) { return f->levels.size(); }

void fused_destroy(Fused* f) { delete f; }

}  // namespace lsw
