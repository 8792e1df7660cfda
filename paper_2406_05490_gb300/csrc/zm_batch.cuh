// zm_batch.cuh -- host-side executor of the batched high-order (FP32C) path, shared by the
// fixed batches of zm_batch_* (zm_batch.cu) and the serving loop (zm_serve.cu).
#pragma once

#include <vector>

#include "zm_internal.cuh"

namespace zm {

// Candidate patch shapes (tp1, tp2) of the 256-node tiles; index 0 is 16 x 16.
constexpr int kNumShapes = 5;
extern const int kShapes[kNumShapes][2];
// Tiles an interface's record buffers hold: enough for any candidate shape.
size_t tile_capacity(int n1, int n2);

class Batch {
public:
    std::vector<Inst> h;  // members: host copy of the device descriptors
    Inst *d = nullptr;    // device descriptors
    int d_cap = 0;
    int *block_inst = nullptr;  // point-kernel block -> member
    int bi_cap = 0;
    int nblocks = 0;
    long long nitems = 0;
    int ctas = 0, occ = 1, sms = 152;
    bool tc = false;  // far pairs: CUDA cores (br32_batch_kernel), or tensor cores (br32tc_kernel)
    int chunk_override = 0;  // 0: default work-item size by mesh size
    int shape = 0;           // index into the candidate patch shapes (0: 16 x 16)
    unsigned long long *counter = nullptr;
    int *err = nullptr;
    std::vector<void *> owned;  // slabs allocated by init() (fixed batches)
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream for graph capture
    cudaGraphExec_t gexec = nullptr;
    Prof own;
    Prof *prof = &own;
    int device = 0;
    std::vector<int> bi_host;

    ~Batch() { release(); }
    void release();

    // Device memory of one interface (one slab).  async: stream-ordered allocation on s.
    static size_t inst_bytes(const zm_mesh &m);
    static int alloc_inst(Inst &I, const zm_mesh &m, double atwood, double g, double mu, double delta,
                          double dt, cudaStream_t s, bool async, void **slab);

    int setup();                    // counters, capture stream, occupancy (once)
    int init(int n, const zm_mesh *meshes, const double *atwood, double g, double mu,
             const double *delta);  // fixed batch owning its slabs
    int plan();                     // (re)build launch plan and descriptors for h
    int set_chunk(int chunk);
    // time candidate work-item sizes on the resident states, keep the fastest
    int autotune(const char *cache_path, int *chosen, float *best_ms);
    // re-tile every member with candidate patch shape k (records cleared, plan rebuilt)
    int set_shape(int k);
    // time candidate patch shapes, then work-item sizes for the best one; keep the fastest
    int autotune_tiles(const char *cache_path, int *shape_out, int *chunk_out, float *best_ms);
    float time_eval(int *rc);  // ms of two derivative evaluations after a warm-up
    int set_dt(double dt);          // all members
    void drop_graph();

    int derivative(int yin, cudaStream_t s);
    int vorticity(int yin, int mode, int yout, double ca, double cb, cudaStream_t s);
    int rk3_step_launches(cudaStream_t s);
    int step(int nsteps, bool use_graph);
    int status();
};

}  // namespace zm
