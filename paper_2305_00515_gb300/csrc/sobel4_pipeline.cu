// sobel4_pipeline.cu — graph-captured video pipeline: per frame slot, one CUDA
// graph of host->device copy and the kernel, which stores the result straight
// into the slot's page-locked host output (no device->host copy), launched on
// the slot's own stream so the upload of one slot overlaps the kernel of
// another.  This is the stream processing that the paper proposes for its
// IO bottleneck (Section 5.2, Section 6).
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <vector>

#include "sobel4.h"
#include "sobel4_launch.h"

namespace {

struct Slot {
  uint8_t *h_in = nullptr;   // pinned
  void *h_out = nullptr;     // pinned
  uint8_t *d_in = nullptr;
  uint8_t *d_out = nullptr;
  unsigned int *d_pair = nullptr;  // the captured kernel's work-queue counter pair (4 words)
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphExec_t kexec = nullptr;  // the slot's kernel alone (caller buffers)
  cudaEvent_t done = nullptr;
  bool pending = false;
  bool out_direct = false;  // exec's kernel stores into h_out itself
};

size_t elem_bytes(int fmt) {
  return fmt == SOBEL4_OUT_F32 ? 4 : ((fmt == SOBEL4_OUT_U8 || fmt == SOBEL4_OUT_EDGE8) ? 1 : 2);
}

}  // namespace

struct sobel4_pipeline_ctx {
  sobel4_handle h = nullptr;
  int device = 0;
  int32_t H = 0, W = 0;
  int border = 0, fmt = 0;
  size_t in_pitch = 0, out_pitch = 0, in_bytes = 0, out_bytes = 0;
  std::vector<Slot> slots;
  int64_t kernels_per_frame = 1;  // kernels in one slot's captured graph
};

namespace {

void release(sobel4_pipeline_ctx *p) {
  for (Slot &s : p->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.kexec) cudaGraphExecDestroy(s.kexec);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.h_in) cudaFreeHost(s.h_in);
    if (s.h_out) cudaFreeHost(s.h_out);
    if (s.d_in) cudaFree(s.d_in);
    if (s.d_out) cudaFree(s.d_out);
    if (s.d_pair) cudaFree(s.d_pair);
  }
  delete p;
}

// Captures the slot's kernel (input s.d_in, output dst at the pipeline's
// output pitch) into *g.
cudaError_t capture(sobel4_pipeline_ctx *p, Slot &s, void *dst, cudaGraph_t *g,
                    sobel4_status *st) {
  *g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  *st = sobel4::run_with_pair(p->h, s.d_in, p->in_pitch, dst, p->out_pitch, p->H, p->W,
                              p->border, p->fmt, s.stream, s.d_pair);
  return cudaStreamEndCapture(s.stream, g);
}

// A graph's roots (nodes without dependencies) and leaves (nodes nothing
// depends on).
cudaError_t ends_of(cudaGraph_t g, std::vector<cudaGraphNode_t> *roots,
                    std::vector<cudaGraphNode_t> *leaves) {
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (e == cudaSuccess && n) e = cudaGraphGetNodes(g, nodes.data(), &n);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    size_t nd = 0, nu = 0;
    e = cudaGraphNodeGetDependencies(nodes[i], nullptr, nullptr, &nd);
    if (e == cudaSuccess) e = cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nu);
    if (e == cudaSuccess && nd == 0) roots->push_back(nodes[i]);
    if (e == cudaSuccess && nu == 0) leaves->push_back(nodes[i]);
  }
  return e;
}

}  // namespace

extern "C" sobel4_status sobel4_pipeline_create(sobel4_handle h, int32_t height, int32_t width,
                                                sobel4_border border, sobel4_format fmt,
                                                int32_t slots, sobel4_pipeline *out) {
  if (!out) return SOBEL4_ERR_INVALID_ARG;
  *out = nullptr;
  if (!h || slots < 2 || slots > 64 || height < 1 || width < 1) return SOBEL4_ERR_INVALID_ARG;
  const int dev = sobel4::handle_info(h).device;
  sobel4::DeviceScope scope(dev);
  sobel4_pipeline_ctx *p = new (std::nothrow) sobel4_pipeline_ctx();
  if (!p) return SOBEL4_ERR_OOM;
  p->h = h;
  p->device = dev;
  p->H = height;
  p->W = width;
  p->border = border;
  p->fmt = fmt;
  p->in_pitch = ((size_t)width + 15) & ~(size_t)15;
  p->out_pitch = ((size_t)width * elem_bytes(fmt) + 15) & ~(size_t)15;
  const size_t planes = fmt == SOBEL4_OUT_S16X4 ? 4 : 1;
  p->in_bytes = p->in_pitch * (size_t)height;
  p->out_bytes = p->out_pitch * (size_t)height * planes;
  p->slots.resize((size_t)slots);
  cudaError_t e = cudaSuccess;
  sobel4_status st = SOBEL4_OK;
  const uint64_t launches0 = sobel4_launch_count(h);
  for (Slot &s : p->slots) {
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s.h_in, p->in_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&s.h_out, p->out_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s.d_in, p->in_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s.d_out, p->out_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s.d_pair, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(s.d_pair, 0, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    // The input's pitch padding is never read; zero it once so the copies move defined bytes.
    e = cudaMemsetAsync(s.d_in, 0, p->in_bytes, s.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
    if (e != cudaSuccess) break;
    // Two captures of the slot's kernel.  kexec: the kernel alone, into the
    // slot's device output (caller frames whose results must be copied out).
    // exec: the upload as a 1-D memcpy node, then the kernel storing straight
    // into the slot's page-locked output (mapped at the same address on the
    // device), so no download; where that memory is not kernel-writable the
    // kernel writes the device output and a download node follows.
    cudaGraph_t g = nullptr;
    e = capture(p, s, s.d_out, &g, &st);
    if (e == cudaSuccess && st == SOBEL4_OK) e = cudaGraphInstantiate(&s.kexec, g, 0);
    if (g) cudaGraphDestroy(g);
    g = nullptr;
    if (e != cudaSuccess || st != SOBEL4_OK) break;
    s.out_direct = sobel4::host_kernel_writable(s.h_out, p->out_pitch, (size_t)height * planes,
                                                (size_t)width * elem_bytes(fmt), elem_bytes(fmt));
    e = capture(p, s, s.out_direct ? s.h_out : s.d_out, &g, &st);
    if (e == cudaSuccess && st == SOBEL4_OK) {
      std::vector<cudaGraphNode_t> roots, leaves;
      e = ends_of(g, &roots, &leaves);
      cudaGraphNode_t copy_in = nullptr, copy_out = nullptr;
      if (e == cudaSuccess)
        e = cudaGraphAddMemcpyNode1D(&copy_in, g, nullptr, 0, s.d_in, s.h_in, p->in_bytes,
                                     cudaMemcpyHostToDevice);
      for (size_t i = 0; i < roots.size() && e == cudaSuccess; ++i)
        e = cudaGraphAddDependencies(g, &copy_in, &roots[i], nullptr, 1);
      if (e == cudaSuccess && !s.out_direct)
        e = cudaGraphAddMemcpyNode1D(&copy_out, g, leaves.data(), leaves.size(), s.h_out,
                                     s.d_out, p->out_bytes, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&s.exec, g, 0);
    }
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || st != SOBEL4_OK) break;
  }
  if (st == SOBEL4_OK && e != cudaSuccess)
    st = e == cudaErrorMemoryAllocation ? SOBEL4_ERR_OOM : SOBEL4_ERR_CUDA;
  if (st != SOBEL4_OK) {
    (void)cudaGetLastError();  // the failure is reported here, not by a later call
    release(p);
    return st;
  }
  // Capturing recorded the kernels into the graphs without launching them.
  // Captures are not launches; each replay launches this many kernels.
  const uint64_t captured = sobel4_launch_count(h) - launches0;
  p->kernels_per_frame = p->slots.empty() ? 1 : (int64_t)(captured / (2 * p->slots.size()));
  sobel4::note_launches(h, -(int64_t)captured);
  *out = p;
  return SOBEL4_OK;
}

extern "C" sobel4_status sobel4_pipeline_buffers(sobel4_pipeline p, int32_t slot, uint8_t **h_in,
                                                 void **h_out, size_t *in_pitch,
                                                 size_t *out_pitch) {
  if (!p || slot < 0 || slot >= (int32_t)p->slots.size()) return SOBEL4_ERR_INVALID_ARG;
  if (h_in) *h_in = p->slots[slot].h_in;
  if (h_out) *h_out = p->slots[slot].h_out;
  if (in_pitch) *in_pitch = p->in_pitch;
  if (out_pitch) *out_pitch = p->out_pitch;
  return SOBEL4_OK;
}

namespace {

// Launches the slot's frame: its graph on its own buffers, else the caller's
// upload, the kernel's graph and the caller's download on the slot's stream.
sobel4_status launch_slot(sobel4_pipeline p, Slot &s, const void *in, void *out) {
  cudaError_t e = cudaSuccess;
  sobel4_status st = SOBEL4_OK;
  bool graph = true;  // the launch replays a captured graph (counted here)
  if (in == s.h_in && out == s.h_out) {
    e = cudaGraphLaunch(s.exec, s.stream);
  } else {
    const size_t planes = p->fmt == SOBEL4_OUT_S16X4 ? 4 : 1;
    e = cudaMemcpyAsync(s.d_in, in, p->in_bytes, cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess &&
        sobel4::host_kernel_writable(out, p->out_pitch, (size_t)p->H * planes,
                                     (size_t)p->W * elem_bytes(p->fmt), elem_bytes(p->fmt))) {
      // the kernel stores the result into the caller's page-locked buffer
      graph = false;
      st = sobel4::run_with_pair(p->h, s.d_in, p->in_pitch, out, p->out_pitch, p->H, p->W,
                                 p->border, p->fmt, s.stream, s.d_pair);
    } else if (e == cudaSuccess) {
      e = cudaGraphLaunch(s.kexec, s.stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, s.d_out, p->out_bytes, cudaMemcpyDeviceToHost, s.stream);
    }
  }
  if (e == cudaSuccess && st == SOBEL4_OK) e = cudaEventRecord(s.done, s.stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    sobel4::note_cuda_error(p->h, e);
    return SOBEL4_ERR_CUDA;
  }
  if (st != SOBEL4_OK) return st;
  s.pending = true;
  if (graph) sobel4::note_launches(p->h, p->kernels_per_frame);
  return SOBEL4_OK;
}

}  // namespace

extern "C" sobel4_status sobel4_pipeline_submit(sobel4_pipeline p, int32_t slot) {
  return sobel4_pipeline_submit_from(p, slot, nullptr, nullptr);
}

extern "C" sobel4_status sobel4_pipeline_submit_from(sobel4_pipeline p, int32_t slot,
                                                     const uint8_t *h_in, void *h_out) {
  if (!p || slot < 0 || slot >= (int32_t)p->slots.size()) return SOBEL4_ERR_INVALID_ARG;
  Slot &s = p->slots[slot];
  if (s.pending) return SOBEL4_ERR_INVALID_ARG;  // wait for the slot before refilling it
  sobel4::DeviceScope scope(p->device);
  return launch_slot(p, s, h_in ? (const void *)h_in : (const void *)s.h_in,
                     h_out ? h_out : s.h_out);
}

extern "C" sobel4_status sobel4_pipeline_wait(sobel4_pipeline p, int32_t slot) {
  if (!p || slot < 0 || slot >= (int32_t)p->slots.size()) return SOBEL4_ERR_INVALID_ARG;
  Slot &s = p->slots[slot];
  if (!s.pending) return SOBEL4_OK;
  sobel4::DeviceScope scope(p->device);
  const cudaError_t e = cudaEventSynchronize(s.done);
  s.pending = false;
  return e == cudaSuccess ? SOBEL4_OK : SOBEL4_ERR_CUDA;
}

extern "C" sobel4_status sobel4_pipeline_destroy(sobel4_pipeline p) {
  if (!p) return SOBEL4_OK;
  sobel4::DeviceScope scope(p->device);
  release(p);
  return SOBEL4_OK;
}
