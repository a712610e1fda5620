// Internal layout of a batch of uneven instances (batch.cu, batch_solve.cu).
#pragma once

#include <string>
#include <vector>

#include "ibem_internal.cuh"

namespace ibem {

struct BatchInst {
    int helm, p, pp, nb, ne1, n1, q, q2, m, R;
    float kappa;
    int64_t E, N, Nstar, C;
    long long lvl[12];
    const double* ext;
    const float* Mf;
    const float* Sf;
    const int64_t* near_ptr;
    const int32_t* near_src;
    const float* near32;
    const int64_t* far_ptr;
    const int32_t* far_src;
    const int32_t* far_rows;
    const float* igeo32;
    float *xs, *ys, *xh, *yh;
    int64_t xoff;
};

}  // namespace ibem

struct ibem_batch {
    int n = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<ibem_handle*> handles;
    std::vector<ibem::BatchInst> inst;
    ibem::BatchInst* d_inst = nullptr;
    std::vector<int64_t> offsets;            // n + 1, in doubles
    int max_m = 0;
    // stage work lists: prefix sums per instance (n + 1 each)
    enum { ST_LIFT, ST_LEAF, ST_BACK, ST_NEAR, ST_RESTRICT, ST_COUPLE, ST_FIXED };
    std::vector<std::vector<int64_t>> pre;   // ST_FIXED fixed stages + 2 per level (m2m, l2l)
    std::vector<int64_t*> d_pre;
    float* arena = nullptr;
    size_t arena_floats = 0;
    size_t yh_begin = 0, yh_floats = 0;      // contiguous y^ region (cleared per application)
    int* d_counter = nullptr;
    int couple_threads = 256;
    int couple_rb = 8;                       // right-hand sides per coupling work item (autotuned)
    std::vector<float> tune_ms;              // autotuner timings, tiles x CTA sizes
    int couple_ctas = 0;
    int launches = 0;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const double* graph_x = nullptr;
    double* graph_y = nullptr;
    double* solve_x = nullptr;               // fixed operator input / output of ibem_batch_solve
    double* solve_y = nullptr;
    std::string err;
};

