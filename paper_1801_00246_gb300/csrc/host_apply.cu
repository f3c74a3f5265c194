// The operator apply on fields in host memory (dg_apply_host): the copies in
// and out run on two copy streams, overlapped with the apply where its
// kernels allow. The tcgen05 FP64 apply (the FP64 default from degree 3) runs
// in chunks of rows: chunk i's gradient product, which reads only its own
// elements' u, starts once chunk i has arrived while later chunks are still
// being copied in; chunk i's neighbour phase and output product follow as soon
// as the gradient products of the chunks holding its neighbours are done, and
// its copy out starts while later chunks are still being computed. Every other
// kernel copies the whole input in, applies and copies the whole result out, in
// order on the caller's stream.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>

#include "dg_internal.h"

using namespace dgx;

namespace {

struct HostCtx {
  dg_mesh* m;
  cudaStream_t st;
  const char* uh;  // host input
  char* oh;        // host output
  char* ud;        // device copies
  char* od;
  size_t row_bytes;  // one element's nodes of one right-hand side
};

// before chunk i's gradient product: copy its rows in on the input stream and
// make the compute stream wait for them
cudaError_t chunk_in(void* c, int i, int64_t r0, int64_t r1) {
  HostCtx* x = static_cast<HostCtx*>(c);
  const size_t off = size_t(r0) * x->row_bytes, n = size_t(r1 - r0) * x->row_bytes;
  cudaError_t e = cudaMemcpyAsync(x->ud + off, x->uh + off, n, cudaMemcpyHostToDevice, x->m->hx_in);
  if (e == cudaSuccess) e = cudaEventRecord(x->m->hx_ev[i], x->m->hx_in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(x->st, x->m->hx_ev[i], 0);
  return e;
}

// after chunk i's output product: copy its rows out on the output stream
cudaError_t chunk_out(void* c, int i, int64_t r0, int64_t r1) {
  HostCtx* x = static_cast<HostCtx*>(c);
  const size_t off = size_t(r0) * x->row_bytes, n = size_t(r1 - r0) * x->row_bytes;
  cudaEvent_t ev = x->m->hx_ev[dg_mesh::kHostChunks + i];
  cudaError_t e = cudaEventRecord(ev, x->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(x->m->hx_outs, ev, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x->oh + off, x->od + off, n, cudaMemcpyDeviceToHost, x->m->hx_outs);
  return e;
}

dg_status fail(cudaError_t err, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(err));
  return err == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
}

}  // namespace

void free_host_apply(dg_mesh* m) {
  cudaFree(m->hx_u);
  cudaFree(m->hx_out);
  m->hx_u = m->hx_out = nullptr;
  m->hx_cap = 0;
  for (cudaEvent_t& ev : m->hx_ev) {
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
  }
  if (m->hx_in) cudaStreamDestroy(m->hx_in);
  if (m->hx_outs) cudaStreamDestroy(m->hx_outs);
  m->hx_in = m->hx_outs = nullptr;
}

extern "C" dg_status dg_apply_host(const dg_mesh* mc, int degree, dg_prec prec, int B, double lambda,
                                   const void* u_host, void* Au_host, void* stream) {
  if (!mc) { set_error("mesh is NULL"); return DG_ERR_ARG; }
  if (B == 0) return DG_OK;
  if (!u_host || !Au_host) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (degree == 0) degree = mc->N;
  if (degree < 1 || degree > kMaxN) { set_error("degree must be in 1..10"); return DG_ERR_ARG; }
  if (prec != DG_F64 && prec != DG_F32 && prec != DG_F64_DFMA) { set_error("bad precision"); return DG_ERR_ARG; }
  if (B < 0 || B > DG_MAX_BATCH) { set_error("batch must be in 0..64"); return DG_ERR_ARG; }
  if (u_host == Au_host) { set_error("u and Au must not alias"); return DG_ERR_ARG; }
  if (!std::isfinite(lambda) || lambda < 0) { set_error("lambda must be finite and >= 0"); return DG_ERR_ARG; }
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  try {
    cudaError_t e = ensure_ops(m, degree);
    if (e != cudaSuccess) return fail(e, "dg_apply_host");
    const int Np = (degree + 1) * (degree + 2) / 2;
    const size_t word = prec == DG_F32 ? sizeof(float) : sizeof(double);
    const int64_t nE = int64_t(B) * m->K;
    const size_t bytes = size_t(nE) * Np * word;
    if (!m->hx_in) {  // copy streams and events, once per mesh
      e = cudaStreamCreateWithFlags(&m->hx_in, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->hx_outs, cudaStreamNonBlocking);
      for (cudaEvent_t& ev : m->hx_ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        free_host_apply(m);
        return fail(e, "dg_apply_host");
      }
    }
    if (m->hx_cap < bytes) {  // device copies of u and Au; cudaFree waits for earlier uses
      cudaFree(m->hx_u);
      cudaFree(m->hx_out);
      m->hx_u = m->hx_out = nullptr;
      m->hx_cap = 0;
      e = cudaMalloc(&m->hx_u, bytes);
      if (e == cudaSuccess) e = cudaMalloc(&m->hx_out, bytes);
      if (e != cudaSuccess) return fail(e, "dg_apply_host");
      m->hx_cap = bytes;
    }
    const bool chunked = prec == DG_F64 && selected_kernel(m, degree, prec, lambda != 0.0) == DG_KERNEL_TC64;
    if (!chunked) {
      e = cudaMemcpyAsync(m->hx_u, u_host, bytes, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = launch_apply(m, degree, prec, B, lambda, m->hx_u, m->hx_out, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(Au_host, m->hx_out, bytes, cudaMemcpyDeviceToHost, st);
      return e == cudaSuccess ? DG_OK : fail(e, "dg_apply_host");
    }
    // chunks of whole waves of 128-row tiles (one tile per SM): one wave first and
    // last (their copies are not overlapped), four in between, at most kHostChunks
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(e, "dg_apply_host");
    const int64_t wave = int64_t(std::max(sms, 1)) * 128;
    int64_t mid = 4 * wave;
    const int64_t minrows = (nE + dg_mesh::kHostChunks - 3) / (dg_mesh::kHostChunks - 2);
    if (mid < minrows) mid = (minrows + 127) / 128 * 128;
    int64_t bounds[dg_mesh::kHostChunks + 1];
    int nch = 0;
    bounds[0] = 0;
    while (bounds[nch] < nE) {
      const int64_t left = nE - bounds[nch];
      // the first chunk and the last one wave; the others leave one wave for the last
      const int64_t take = (nch == 0 || left <= wave) ? std::min(left, wave) : std::min(mid, left - wave);
      bounds[nch + 1] = bounds[nch] + take;
      ++nch;
    }
    // the copies in start after the caller's earlier work (which may still read the
    // device copy of u); the caller's later work starts after the last copy out
    cudaEvent_t ev_start = m->hx_ev[2 * dg_mesh::kHostChunks], ev_done = m->hx_ev[2 * dg_mesh::kHostChunks + 1];
    e = cudaEventRecord(ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m->hx_in, ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m->hx_outs, ev_start, 0);
    if (e != cudaSuccess) return fail(e, "dg_apply_host");
    HostCtx ctx{m, st, static_cast<const char*>(u_host), static_cast<char*>(Au_host), static_cast<char*>(m->hx_u),
                static_cast<char*>(m->hx_out), size_t(Np) * word};
    ApplyChunks ch;
    ch.n = nch;
    ch.bounds = bounds;
    ch.before = chunk_in;
    ch.after = chunk_out;
    ch.ctx = &ctx;
    e = launch_apply_tc64(m, degree, B, lambda, static_cast<const double*>(m->hx_u), static_cast<double*>(m->hx_out),
                          st, nullptr, &ch);
    // join the copy streams back into the caller's stream, also after a failed launch
    const cudaError_t e2 = cudaEventRecord(ev_done, m->hx_outs);
    const cudaError_t e3 = e2 == cudaSuccess ? cudaStreamWaitEvent(st, ev_done, 0) : e2;
    if (e == cudaSuccess) e = e3;
    return e == cudaSuccess ? DG_OK : fail(e, "dg_apply_host");
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return DG_ERR_OOM;
  }
}
