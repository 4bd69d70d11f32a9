// bp.cuh -- learned-potential (Behler-Parrinello) argument blocks.
#pragma once

#include "kernels.cuh"

namespace jmd {

constexpr float BP_RC = 3.77f;     // descriptor cutoff (A)
constexpr float BP_ETA_R = 8.0f;   // radial width (A^-2)
constexpr float BP_ETA_A = 0.05f;  // angular width (A^-2)
constexpr int BP_H = 64;           // hidden width
constexpr int BP_D = 16;           // descriptors per atom

// Packed FP32 parameter vector: W1 [64][16], b1 [64], W2 [64][64], b2 [64],
// w3 [64], b3 [1]  (5,313 values).
constexpr int P_W1 = 0, P_B1 = 1024, P_W2 = 1088, P_B2 = 5184, P_W3 = 5248, P_B3 = 5312, P_TOTAL = 5313;

struct BpArgs {
    Box box;
    int N, cap;
    int sys_n;           // atoms per system when several equal-size systems are concatenated
                         // (rows hold indices local to the system); 0 = one system
    const float4 *r;
    const int32_t *nbr, *cnt;
    float *G;            // [N][16] descriptors (out of k_bp_desc)
    const float *dEdG;   // [N][16] network input gradient
    const float *Ei;     // [N] per-atom network energies (may be NULL)
    const float4 *dF;    // [N] vector field for the descriptor JVP
    float *V;            // [N][16] JVP output
    uint32_t *status;
    PairArgs pa;         // forces out (pa.f), optional kick and energy reductions
};

void enqueue_bp_desc(const BpArgs &a, cudaStream_t st);
void enqueue_bp_force(const BpArgs &a, int kick, cudaStream_t st);
void enqueue_bp_jvp(const BpArgs &a, cudaStream_t st);
// descriptors and the tcgen05 network in one kernel (mlp_tc.cu): Ei, dE/dG
void enqueue_bp_desc_mlp_tc(const BpArgs &b, const float *P, const float *norm, float *Ei, float *dEdG,
                            uint32_t *status, cudaStream_t st);
size_t mlp_train_tc_scratch(int N);   // partial gradients of md_bp_mlp_train_tc

}  // namespace jmd
