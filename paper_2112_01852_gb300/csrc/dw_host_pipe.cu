// Host-buffer apply in time slabs (dw_apply_host).
//
// The operators couple a site only to its t +- 1 neighbours (Sec. 4.1: the
// hopping term is nearest-neighbour in 4D, the fifth-dimension terms are local
// in x), so the field can be moved through the device slab by slab: while slab
// k+1 is copied in, the operator runs on slab k and slab k-1 is copied out.
// Three streams carry the copies in, the stencil launches and the copies out;
// events order them.  The operator on a slab starts once the slab and both t
// neighbours are resident; for D^+D the second pass on a slab waits for the
// first pass on the slab and its neighbours.  With the blocked fermion layout
// a t slab is one contiguous byte range per right-hand side when Lx Ly Lz is a
// multiple of the 32-site block.
#include <algorithm>
#include <vector>

#include "dw_api_internal.cuh"

namespace dw {

namespace {

struct Task {
  int pass;   // 0: first operator (or the only one), 1: D^+ of D^+D
  int slab;
  int wait_in;  // copy-in event the task waits for (-1: none)
};

int pipe_streams(dw_lattice *lat) {
  if (lat->pipe_in) return DW_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&lat->pipe_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&lat->pipe_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline stream creation");
  return DW_OK;
}

int pipe_events(dw_lattice *lat, size_t n) {
  while (lat->pipe_events.size() < n) {
    cudaEvent_t ev;
    const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline event creation");
    lat->pipe_events.push_back(ev);
  }
  return DW_OK;
}

// Number of slabs: the largest divisor of Lt that is at most kMaxSlabs and
// leaves slabs of at least kMinSlabSites 4D sites (smaller launches do not
// fill the GPU).
constexpr int kMaxSlabs = 64;
constexpr long long kMinSlabSites = 8192;

int slab_count(const dw_lattice *lat) {
  const long long Vs = (long long)lat->dims[0] * lat->dims[1] * lat->dims[2];
  if (Vs % 32) return 1;
  int best = 1;
  for (int n = 2; n <= kMaxSlabs && n <= lat->dims[3]; ++n)
    if (lat->dims[3] % n == 0 && Vs * (lat->dims[3] / n) >= kMinSlabSites) best = n;
  return best;
}

int run_pass(dw_lattice *lat, int op, int pass, void *out, const void *in, void *mid,
             const double *mf, int nrhs, cudaStream_t st, int t0, int nt) {
  const int prec = lat->prec;
  switch (op) {
    case DW_OP_DHOP:
      return run_dslash(lat, prec, OP_DHOP, out, in, nullptr, nrhs, st, nullptr, nullptr, 0,
                        nullptr, nullptr, nullptr, t0, nt);
    case DW_OP_DHOP_DAG:
      return run_dslash(lat, prec, OP_DHOP_DAG, out, in, nullptr, nrhs, st, nullptr, nullptr, 0,
                        nullptr, nullptr, nullptr, t0, nt);
    case DW_OP_D:
      return run_dslash(lat, prec, OP_D, out, in, mf, nrhs, st, nullptr, nullptr, 0, nullptr,
                        nullptr, nullptr, t0, nt);
    case DW_OP_DDAG:
      return run_dslash(lat, prec, OP_DDAG, out, in, mf, nrhs, st, nullptr, nullptr, 0, nullptr,
                        nullptr, nullptr, t0, nt);
    case DW_OP_DDAGD:
      if (pass == 0)
        return run_dslash(lat, prec, OP_D, mid, in, mf, nrhs, st, nullptr, nullptr, 0, nullptr,
                          nullptr, nullptr, t0, nt);
      return run_dslash(lat, prec, OP_DDAG, out, mid, mf, nrhs, st, nullptr, nullptr, 0, nullptr,
                        nullptr, nullptr, t0, nt);
  }
  return fail(DW_ERR_ARG, "unknown operator %d", op);
}

// Order of the operator launches on the compute stream.  Pass 0 on slab k
// needs the copies of slabs k-1, k, k+1 (mod n); the copies arrive in slab
// order, so it waits for the copy of the highest of the three and the tasks
// are sorted by that.  Pass 1 on slab k follows the last of pass 0 on k-1, k,
// k+1 in this order.
std::vector<Task> schedule(int n, int passes) {
  std::vector<Task> first;
  for (int k = 0; k < n; ++k) {
    const int w = std::max(k, std::max((k + n - 1) % n, (k + 1) % n));
    first.push_back({0, k, w});
  }
  std::stable_sort(first.begin(), first.end(),
                   [](const Task &a, const Task &b) { return a.wait_in < b.wait_in; });
  if (passes == 1) return first;
  std::vector<int> pos(n);
  for (int i = 0; i < n; ++i) pos[first[i].slab] = i;
  std::vector<std::vector<int>> after(n);  // pass-1 slabs released by first[i]
  for (int k = 0; k < n; ++k) {
    const int last = std::max(pos[k], std::max(pos[(k + n - 1) % n], pos[(k + 1) % n]));
    after[last].push_back(k);
  }
  std::vector<Task> all;
  for (int i = 0; i < n; ++i) {
    all.push_back(first[i]);
    for (int k : after[i]) all.push_back({1, k, -1});
  }
  return all;
}

}  // namespace

int apply_host_pipelined(dw_lattice *lat, int op, void *out_host, const void *in_host,
                         const double *mf, int nrhs, cudaStream_t st) {
  const int n = slab_count(lat);
  const size_t rhs_bytes = field_bytes(lat, lat->prec, 1);
  const size_t bytes = rhs_bytes * (size_t)nrhs;
  size_t cap_in = lat->stage_bytes, cap_out = lat->stage_bytes;
  int rc = ensure_buffer(&lat->stage_in, &cap_in, bytes);
  if (rc) return rc;
  rc = ensure_buffer(&lat->stage_out, &cap_out, bytes);
  if (rc) return rc;
  lat->stage_bytes = cap_in < cap_out ? cap_in : cap_out;
  void *mid = nullptr;
  if (op == DW_OP_DDAGD) {
    rc = ensure_buffer(&lat->scratch, &lat->scratch_bytes, bytes);
    if (rc) return rc;
    mid = lat->scratch;
  }
  if (n == 1) {  // one slab: copy in, apply, copy out on the caller's stream
    cudaError_t e = cudaMemcpyAsync(lat->stage_in, in_host, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    rc = apply_op(lat, op, lat->stage_out, lat->stage_in, mf, nrhs, st);
    if (rc) return rc;
    e = cudaMemcpyAsync(out_host, lat->stage_out, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? DW_OK : cuda_fail(e, "stream synchronize");
  }
  rc = pipe_streams(lat);
  if (rc) return rc;
  const int passes = op == DW_OP_DDAGD ? 2 : 1;
  const std::vector<Task> tasks = schedule(n, passes);
  // events: [0, n) copies in, [n, n + tasks) operator launches, then one for
  // the caller's stream
  rc = pipe_events(lat, (size_t)n + tasks.size() + 1);
  if (rc) return rc;
  cudaEvent_t *ev = lat->pipe_events.data();
  cudaEvent_t ev_start = ev[n + tasks.size()];
  const int T = lat->dims[3] / n;
  const size_t slab_bytes = rhs_bytes / (size_t)n;  // Vs % 32 == 0: no padding, equal slabs
  // one plain copy per right-hand side (a field can exceed the largest pitch
  // a 2D copy accepts)
  auto copy = [&](void *dst, const void *src, int k, cudaMemcpyKind kind, cudaStream_t s) {
    for (int r = 0; r < nrhs; ++r) {
      const size_t off = (size_t)r * rhs_bytes + (size_t)k * slab_bytes;
      const cudaError_t ce =
          cudaMemcpyAsync((char *)dst + off, (const char *)src + off, slab_bytes, kind, s);
      if (ce != cudaSuccess) return ce;
    }
    return cudaSuccess;
  };
  // on an error after work was queued, let it drain before the host buffers
  // go back to the caller
  auto bail = [&](int code) {
    cudaStreamSynchronize(lat->pipe_in);
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(lat->pipe_out);
    return code;
  };
  // the staging buffers may still be read by earlier work on the caller's stream
  cudaError_t e = cudaEventRecord(ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(lat->pipe_in, ev_start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(lat->pipe_out, ev_start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline ordering");
  for (int k = 0; k < n; ++k) {
    e = copy(lat->stage_in, in_host, k, cudaMemcpyHostToDevice, lat->pipe_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev[k], lat->pipe_in);
    if (e != cudaSuccess) return bail(cuda_fail(e, "host-to-device copy"));
  }
  for (size_t i = 0; i < tasks.size(); ++i) {
    const Task &t = tasks[i];
    if (t.wait_in >= 0) {
      e = cudaStreamWaitEvent(st, ev[t.wait_in], 0);
      if (e != cudaSuccess) return bail(cuda_fail(e, "pipeline ordering"));
    }
    rc = run_pass(lat, op, t.pass, lat->stage_out, lat->stage_in, mid, mf, nrhs, st,
                  t.slab * T, T);
    if (rc) return bail(rc);
    e = cudaEventRecord(ev[n + i], st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "pipeline ordering"));
    if (t.pass == passes - 1) {  // the slab is final: copy it out
      e = cudaStreamWaitEvent(lat->pipe_out, ev[n + i], 0);
      if (e == cudaSuccess) e = copy(out_host, lat->stage_out, t.slab, cudaMemcpyDeviceToHost,
                                     lat->pipe_out);
      if (e != cudaSuccess) return bail(cuda_fail(e, "device-to-host copy"));
    }
  }
  e = cudaStreamSynchronize(lat->pipe_out);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? DW_OK : cuda_fail(e, "stream synchronize");
}

void pipe_release(dw_lattice *lat) {
  for (cudaEvent_t ev : lat->pipe_events) cudaEventDestroy(ev);
  lat->pipe_events.clear();
  if (lat->pipe_in) cudaStreamDestroy(lat->pipe_in);
  if (lat->pipe_out) cudaStreamDestroy(lat->pipe_out);
  lat->pipe_in = lat->pipe_out = nullptr;
}

}  // namespace dw
