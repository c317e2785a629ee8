// CUDA-graph capture of H_eff psi for one or many contexts.
//
// The H_eff psi of each context is a memset of sigma plus its prepared
// grouped-GEMM launches; capturing them once turns every later product into a
// single graph launch (no per-launch CPU cost, no gaps between the chunks).
// Several contexts (independent problems) are captured as parallel branches
// of one graph, so all their blocks share the GPU in one replay.
#include <cuda_runtime.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "engine.hpp"
#include "graph.hpp"

namespace qd {

#define GK(x)                                                                                  \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) throw std::runtime_error(std::string("CUDA: ") + cudaGetErrorString(e_)); \
  } while (0)

struct HeffGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  cudaStream_t cap = nullptr;
  double flops = 0;
  int nodes = 0;
};

HeffGraph* graph_create(const std::vector<Engine*>& eng, const std::vector<uint64_t>& psi,
                        const std::vector<uint64_t>& sig, int prec) {
  auto* G = new HeffGraph();
  try {
    const size_t n = eng.size();
    GK(cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking));
    G->side.resize(n);
    G->ev.resize(n + 1);
    for (size_t i = 0; i < n; ++i) GK(cudaStreamCreateWithFlags(&G->side[i], cudaStreamNonBlocking));
    for (auto& e : G->ev) GK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // one eager run first: lazily initialised kernel attributes are set
    // outside the capture
    for (size_t i = 0; i < n; ++i) {
      eng[i]->heff(psi[i], sig[i], G->cap, prec);
      G->flops += eng[i]->plan.flops;
    }
    GK(cudaStreamSynchronize(G->cap));
    GK(cudaStreamBeginCapture(G->cap, cudaStreamCaptureModeThreadLocal));
    GK(cudaEventRecord(G->ev[n], G->cap));
    for (size_t i = 0; i < n; ++i) {
      GK(cudaStreamWaitEvent(G->side[i], G->ev[n], 0));
      eng[i]->heff(psi[i], sig[i], G->side[i], prec);
      GK(cudaEventRecord(G->ev[i], G->side[i]));
      GK(cudaStreamWaitEvent(G->cap, G->ev[i], 0));
    }
    GK(cudaStreamEndCapture(G->cap, &G->g));
    size_t nn = 0;
    GK(cudaGraphGetNodes(G->g, nullptr, &nn));
    G->nodes = (int)nn;
    GK(cudaGraphInstantiate(&G->x, G->g, 0));
  } catch (...) {
    cudaStreamCaptureStatus st;
    if (G->cap && cudaStreamIsCapturing(G->cap, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(G->cap, &junk);
      if (junk) cudaGraphDestroy(junk);
    }
    graph_destroy(G);
    throw;
  }
  return G;
}

void graph_launch(HeffGraph* G, void* stream) { GK(cudaGraphLaunch(G->x, (cudaStream_t)stream)); }

double graph_flops(const HeffGraph* G) { return G->flops; }
int graph_nodes(const HeffGraph* G) { return G->nodes; }

void graph_destroy(HeffGraph* G) {
  if (!G) return;
  if (G->x) cudaGraphExecDestroy(G->x);
  if (G->g) cudaGraphDestroy(G->g);
  for (auto s : G->side)
    if (s) cudaStreamDestroy(s);
  for (auto e : G->ev)
    if (e) cudaEventDestroy(e);
  if (G->cap) cudaStreamDestroy(G->cap);
  delete G;
}

}  // namespace qd
