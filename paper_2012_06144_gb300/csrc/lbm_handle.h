// lbm_handle.h -- the simulation handle behind the opaque lbm_t of the C ABI
// (shared by the single-simulation entry points and the batch).
#pragma once

#include <cstdint>
#include <string>

#include "lbm.h"
#include "lbm_internal.h"

struct lbm_t {
    lbm_domain dom;
    lbm_params prm;
    lbm::Params kp;
    cudaStream_t stream;
    int device;
    char *ws;
    size_t ws_bytes;
    bool owns_ws;
    lbm::Storage sto;
    bool unfused;      // LBM_FORM_UNFUSED: natural two-grid storage, Algorithm 1's passes
    lbm::Unfused uf;
    float *phi[2];
    int *flag;
    double *red_scratch, *red_out;
    int cur;      // phi[cur] holds phi^t
    int64_t t;    // time level: steps advanced since initialisation
    bool ready;   // a state exists
    std::string err;
    // runs of kStepGraph steps of small boxes replayed from CUDA graphs, by the
    // AA parity of the first step and the phi buffer it reads ((t & 1) * 2 + cur)
    cudaGraphExec_t step_graph[4];
};

namespace lbm {
// Bookkeeping of one time step advanced by a launch made elsewhere (the batch).
inline void advance_level(lbm_t *s) {
    s->cur ^= 1;
    s->t += 1;
}
}  // namespace lbm
