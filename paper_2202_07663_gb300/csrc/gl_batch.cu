// gl_batch.cu - continuous batching: one CUDA graph, replayed per batch, that
// evaluates log-likelihood + gradient for many (system, vector range)
// segments at once.
//
// The batcher owns a scratch arena (per-vector constants, image work buffers,
// tile partials of every segment of a batch), a device segment table and two
// pinned host staging buffers. The kernel sequence is captured into a graph
// once, with persistent grids that read the segment counts from the device
// table when they run; each batch copies its table into the device (stream
// ordered) and replays the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/gigalens.h"
#include "gl_device.cuh"
#include "gl_internal.h"
#include "gl_launch.h"

namespace {

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Hooks used while capturing: no event records inside the graph.
struct CaptureHooks final : gl::Hooks {
  void before(int, cudaStream_t) override {}
  cudaError_t after(int, cudaStream_t) override { return cudaGetLastError(); }
};

size_t segment_scratch(const gl::Seg& g) {
  return align256(sizeof(gl::VecConst) * size_t(g.B)) + align256(sizeof(float) * size_t(g.B) * g.H * g.W) +
         align256(sizeof(double) * size_t(g.B) * g.ntiles * gl::NACC);
}

}  // namespace

struct gl_batcher {
  int device = 0;
  int max_segments = 0;
  size_t arena_bytes = 0;
  unsigned char* d_arena = nullptr;
  unsigned char* d_table = nullptr;       // TableHdr + Seg[max_segments]
  unsigned char* h_stage[2] = {nullptr, nullptr};
  cudaEvent_t staged[2] = {nullptr, nullptr};
  int slot = 0;
  size_t conv_smem[gl::N_CONV_CLASSES] = {0, 0, 0};
  int max_H = 0, max_W = 0, max_K = 0;
  cudaStream_t capture_stream = nullptr;
  // the last run's graph and its stream: a run on another stream waits for
  // it before it overwrites the device table and the arena that graph reads
  cudaEvent_t done = nullptr;
  cudaStream_t last_stream = nullptr;
  bool ran = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t table_bytes() const { return align256(sizeof(gl::TableHdr)) + sizeof(gl::Seg) * size_t(max_segments); }
};

extern "C" {

int gl_batcher_destroy(gl_batcher* b) {
  if (!b) return GL_OK;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->done) cudaEventDestroy(b->done);
  for (int i = 0; i < 2; ++i) {
    if (b->staged[i]) cudaEventDestroy(b->staged[i]);
    if (b->h_stage[i]) cudaFreeHost(b->h_stage[i]);
  }
  cudaFree(b->d_table);
  cudaFree(b->d_arena);
  delete b;
  return GL_OK;
}

int gl_batcher_create(gl_batcher** out, int max_segments, size_t arena_bytes, int max_H, int max_W, int max_K) {
  if (!out) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null out");
  *out = nullptr;
  if (max_segments < 1 || max_segments > GL_MAX_SEGMENTS)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "max_segments outside [1, GL_MAX_SEGMENTS]");
  if (arena_bytes < (size_t(1) << 20)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "arena below 1 MiB");
  if (max_H < 1 || max_W < 1 || max_K < 1 || (max_K % 2) == 0 || max_K > 63)
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad max_H, max_W or max_K");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gl_internal::cuda_error(e, "cudaGetDevice");
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  gl_batcher* b = new gl_batcher();
  b->device = dev;
  b->max_segments = max_segments;
  b->arena_bytes = arena_bytes;
  b->max_H = max_H;
  b->max_W = max_W;
  b->max_K = max_K;
  // dynamic shared memory per convolution class: largest image, largest PSF of the class
  const int Ks[gl::N_CONV_CLASSES] = {11, 21, max_K};
  for (int c = 0; c < gl::N_CONV_CLASSES; ++c) {
    const int K = Ks[c];
    if (c < 2 && K > max_K) continue;
    size_t one = gl::conv_smem_bytes(max_H, max_W, K, false), two = gl::conv_smem_bytes(max_H, max_W, K, true);
    size_t sm = gl::conv_two_buf(max_H, max_W, K) ? two : one;
    b->conv_smem[c] = sm;
    if (one + 2048 > size_t(optin)) {
      gl_batcher_destroy(b);
      return gl_internal::set_error(GL_ERR_UNSUPPORTED, "max image too large for the shared-memory convolution");
    }
  }
  const size_t tb = b->table_bytes();
  if ((e = cudaMalloc(&b->d_arena, arena_bytes)) != cudaSuccess || (e = cudaMalloc(&b->d_table, tb)) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_stage[0], tb)) != cudaSuccess || (e = cudaMallocHost(&b->h_stage[1], tb)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->staged[0], cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->staged[1], cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    gl_batcher_destroy(b);
    return gl_internal::cuda_error(e, "gl_batcher_create allocation");
  }
  std::memset(b->h_stage[0], 0, tb);
  if ((e = cudaMemcpy(b->d_table, b->h_stage[0], tb, cudaMemcpyHostToDevice)) != cudaSuccess) {
    gl_batcher_destroy(b);
    return gl_internal::cuda_error(e, "table init");
  }
  // capture the kernel sequence once (kernel attributes are set before capture)
  if ((e = gl::prepare_devtable(b->conv_smem)) != cudaSuccess) {
    gl_batcher_destroy(b);
    return gl_internal::cuda_error(e, "kernel attributes");
  }
  CaptureHooks hk;
  const gl::TableHdr* hdr = reinterpret_cast<const gl::TableHdr*>(b->d_table);
  const gl::Seg* segs = reinterpret_cast<const gl::Seg*>(b->d_table + align256(sizeof(gl::TableHdr)));
  e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = gl::launch_devtable(hdr, segs, b->conv_smem, b->capture_stream, &hk);
    e = cudaStreamEndCapture(b->capture_stream, &b->graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    gl_batcher_destroy(b);
    return gl_internal::cuda_error(e, "graph capture of the batched launch");
  }
  *out = b;
  return GL_OK;
}

size_t gl_batcher_segment_bytes(const gl_system* sys, int B) {
  if (!sys || B <= 0) return 0;
  return segment_scratch(gl_internal::seg_without_scratch(sys, nullptr, B));
}

int gl_batcher_run(gl_batcher* b, gl_system* const* systems, const float* const* params, const int* B,
                   double* const* loglik_out, double* const* chi2_out, double* const* grad_out, int n, void* stream) {
  if (!b) return gl_internal::set_error(GL_ERR_INVALID_ARG, "null batcher");
  if (n < 0 || n > b->max_segments) return gl_internal::set_error(GL_ERR_INVALID_ARG, "n outside [0, max_segments]");
  if (n > 0 && (!systems || !params || !B || !loglik_out || !grad_out))
    return gl_internal::set_error(GL_ERR_INVALID_ARG, "null array");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gl_internal::cuda_error(e, "cudaGetDevice");
  if (dev != b->device) return gl_internal::set_error(GL_ERR_INVALID_ARG, "the batcher lives on another device");
  std::vector<gl::Seg> by_class[gl::N_CONV_CLASSES];
  size_t used = 0;
  for (int i = 0; i < n; ++i) {
    if (!systems[i] || B[i] < 0 || B[i] > (1 << 24)) return gl_internal::set_error(GL_ERR_INVALID_ARG, "bad segment");
    if (B[i] == 0) continue;
    const int rc = gl_internal::system_device_check(systems[i]);
    if (rc != GL_OK) return rc;
    if (!params[i] || !loglik_out[i] || !grad_out[i])
      return gl_internal::set_error(GL_ERR_INVALID_ARG, "null params/loglik/grad of a segment");
    gl::Seg g = gl_internal::seg_without_scratch(systems[i], params[i], B[i]);
    if (g.H > b->max_H || g.W > b->max_W || g.K > b->max_K)
      return gl_internal::set_error(GL_ERR_UNSUPPORTED, "segment image or PSF larger than the batcher was built for");
    const int c = gl::conv_class(g.K);
    if (g.conv_sep && gl::seg_conv_smem(g) > b->conv_smem[c]) g.conv_sep = 0;
    if (g.conv_two_buf && gl::conv_smem_bytes(g.H, g.W, g.K, true) > b->conv_smem[c]) g.conv_two_buf = 0;
    if (gl::seg_conv_smem(g) > b->conv_smem[c])
      return gl_internal::set_error(GL_ERR_UNSUPPORTED, "segment convolution does not fit the captured shared memory");
    const size_t need = segment_scratch(g);
    if (used + need > b->arena_bytes) {
      char msg[160];
      snprintf(msg, sizeof(msg), "batch needs more than the %zu-byte scratch arena", b->arena_bytes);
      return gl_internal::set_error(GL_ERR_BUDGET, msg);
    }
    unsigned char* base = b->d_arena + used;
    g.vc = reinterpret_cast<gl::VecConst*>(base);
    g.work = reinterpret_cast<float*>(base + align256(sizeof(gl::VecConst) * size_t(g.B)));
    g.partial = reinterpret_cast<double*>(base + align256(sizeof(gl::VecConst) * size_t(g.B)) +
                                          align256(sizeof(float) * size_t(g.B) * g.H * g.W));
    used += need;
    g.loglik = loglik_out[i];
    g.chi2 = chi2_out ? chi2_out[i] : nullptr;
    g.grad = grad_out[i];
    by_class[c].push_back(g);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int nonempty = 0;
  for (int c = 0; c < gl::N_CONV_CLASSES; ++c) nonempty += int(by_class[c].size());
  if (nonempty == 1) {
    // One segment (the common case of a lightly loaded server): the launch
    // sequence of a single-system call, tuned for its batch size (tile plan,
    // adjoint blocks per SM, small-batch convolution), on its share of the
    // arena; no table, no graph.
    gl::Seg g;
    for (int c = 0; c < gl::N_CONV_CLASSES; ++c)
      if (!by_class[c].empty()) g = by_class[c][0];
    g.conv_two_buf = gl::conv_two_buf(g.H, g.W, g.K) ? 1 : 0;
    g.conv_sep = gl::conv_sep_ok(g.H, g.W, g.K, g.psf_rank) ? 1 : 0;
    if (b->ran && st != b->last_stream && (e = cudaStreamWaitEvent(st, b->done, 0)) != cudaSuccess)
      return gl_internal::cuda_error(e, "wait for the previous run");
    if ((e = gl::launch_one(g, gl::MODE_GRAD, st, gl_internal::hooks())) != cudaSuccess)
      return gl_internal::cuda_error(e, "kernel launch");
    if ((e = cudaEventRecord(b->done, st)) != cudaSuccess) return gl_internal::cuda_error(e, "run event");
    b->last_stream = st;
    b->ran = true;
    return GL_OK;
  }
  // stage the table (wait until the previous copy out of this staging buffer has run)
  const int s = b->slot;
  b->slot ^= 1;
  e = cudaEventSynchronize(b->staged[s]);
  if (e != cudaSuccess) return gl_internal::cuda_error(e, "staging event");
  gl::TableHdr* hdr = reinterpret_cast<gl::TableHdr*>(b->h_stage[s]);
  gl::Seg* segs = reinterpret_cast<gl::Seg*>(b->h_stage[s] + align256(sizeof(gl::TableHdr)));
  std::memset(hdr, 0, sizeof(gl::TableHdr));
  int k = 0, vt = 0, rt = 0;
  for (int c = 0; c < gl::N_CONV_CLASSES; ++c) {
    hdr->conv_first[c] = k;
    int ct = 0;
    for (gl::Seg& g : by_class[c]) {
      g.vec_begin = vt;
      g.ray_begin = rt;
      g.conv_begin = ct;
      vt += g.B;
      rt += g.B * g.ntiles;
      ct += g.B;
      segs[k++] = g;
    }
    hdr->conv_nseg[c] = k - hdr->conv_first[c];
    hdr->conv_total[c] = ct;
  }
  hdr->nseg = k;
  hdr->vec_total = vt;
  hdr->ray_total = rt;
  if (k == 0) return GL_OK;
  const size_t bytes = align256(sizeof(gl::TableHdr)) + sizeof(gl::Seg) * size_t(k);
  if (b->ran && st != b->last_stream && (e = cudaStreamWaitEvent(st, b->done, 0)) != cudaSuccess)
    return gl_internal::cuda_error(e, "wait for the previous run");
  if ((e = cudaMemcpyAsync(b->d_table, b->h_stage[s], bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return gl_internal::cuda_error(e, "table upload");
  if ((e = cudaEventRecord(b->staged[s], st)) != cudaSuccess) return gl_internal::cuda_error(e, "staging event");
  if ((e = cudaGraphLaunch(b->exec, st)) != cudaSuccess) return gl_internal::cuda_error(e, "graph launch");
  if ((e = cudaEventRecord(b->done, st)) != cudaSuccess) return gl_internal::cuda_error(e, "run event");
  b->last_stream = st;
  b->ran = true;
  gl_internal::count_launches(gl::DEVTABLE_LAUNCHES);
  return GL_OK;
}

}  // extern "C"
