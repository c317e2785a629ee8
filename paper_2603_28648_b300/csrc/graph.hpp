// CUDA-graph capture of H_eff psi over one or many engines.
#pragma once
#include <cstdint>
#include <vector>

namespace qd {
struct Engine;
struct HeffGraph;
HeffGraph* graph_create(const std::vector<Engine*>& eng, const std::vector<uint64_t>& psi,
                        const std::vector<uint64_t>& sig, int prec);
void graph_launch(HeffGraph* g, void* stream);
double graph_flops(const HeffGraph* g);
int graph_nodes(const HeffGraph* g);
void graph_destroy(HeffGraph* g);
}  // namespace qd
