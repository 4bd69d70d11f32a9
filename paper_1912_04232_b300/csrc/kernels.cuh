// kernels.cuh -- argument blocks and enqueue functions shared between the
// libjmd translation units (host side).
#pragma once

#include <functional>

#include "common.cuh"

namespace jmd {

struct NbrArgs {
    Box box;
    int N, cap, dim;
    int nc[3];
    float cell_scale[3];
    float r_list2;
    const float4 *r;
    int32_t *nbr, *cnt;
    uint16_t *lrow;  // local rows (MD_NBR_LOCAL_ROWS) or NULL
    float4 *rref;
    WsPtrs ws;
    uint32_t *status;
    const float4 *r_alt;  // fused NVE: positions alternate between r and r_alt by the parity of ctl[CTL_STEP]
    int gated;       // 1: run only if ctl[CTL_REBUILD] != 0
    int canonical;   // 1: sort every row ascending after the build
    int wrapped;     // 1: positions are inside [0, L) (integrators), enabling the wrap-free path
};

struct PairArgs {
    Box box;
    int N, cap, tpp;
    int opt;                // kernel variant: bit 0 stream rows past L1
    const float4 *r;
    const int32_t *nbr, *cnt;
    float4 *f;
    float4 *v;              // KICK only
    float half_dt_over_m;   // KICK only
    float mass;             // KICK only (kinetic energy)
    // fused NVE step (KICK == 2): the next kick-drift into the other buffer
    float4 *r_alt;          // positions alternate between r and r_alt by the parity of ctl[CTL_STEP]
    const float4 *rref;     // positions at the last build (displacement check)
    float dt, half_skin2;
    unsigned long long cond_if;   // graph IF handle of the rebuild chain (0: none)
    // LJ
    float rc2, sigma2, c24eps, c4eps, e_shift;
    // soft sphere
    float eps, alpha;
    // Stillinger-Weber {eps, sigma, a, lambda, gamma, A, B, p, q, cos0, rc, rc2}
    float sw[12];
    // three-body partner lists (tb_layout; SW_LIST_SLOTS slots for
    // Stillinger-Weber, BP_LIST_SLOTS for the learned potential; null: the
    // force kernel tests the neighbors' rows itself)
    int32_t *tb_cnt, *tb_idx;
    float4 *tb_vec;
    float4 *tb_aux, *tb_f2;   // Stillinger-Weber: (g, g', 1/r) per slot, two-body (F, e) per atom
    // learned potential: network and per-atom scratch (device pointers)
    const float *bp_params, *bp_norm;
    float *bp_G, *bp_dEdG, *bp_Ei;
    int bp_sys_n;
    // graph-network potential: the model descriptor by value (so a cached
    // graph's key covers its device pointers)
    md_gnn_model gnn;
    // library switches that change which kernels are enqueued (tensor cores
    // for the networks, atoms per warp): part of every cached graph's key
    int variant;
    // cell-centred path (lists with local rows): 16-bit rows and the cell list
    const uint16_t *lrow;
    const int32_t *atoms, *cell_start;
    int nc[3], ncell, max_blocks;
    // Nose-Hoover chain (nhc.cuh): thermostat state, chain length, series of
    // the conserved extended energy
    double *nhc;
    int nhc_M;
    double *H_out;
    // reductions
    double *E_out, *KE_out;
    int series;             // 1: write E_out[ctl[CTL_STEP]] and advance the counter
    uint32_t *ctl;
    double2 *partials;
    uint32_t *status;
    // device-side loop control inside a CUDA graph WHILE node: the last
    // block sets the loop condition to (step + 1 < ctl[CTL_NSTEPS])
    unsigned long long cond_while;
    int use_cond;
};

NbrArgs make_nbr_args(const md_space *s, const float *d_r, const md_nbr *nb, uint32_t *d_status, int gated);

// Graph loops (graphloop.cu): WHILE(iteration < niter) { body } as one CUDA
// graph; inside the body, rebuild_if() adds the rebuild chain under an IF
// node taken from the device rebuild flag.
struct LoopBuilder {
    cudaGraph_t graph = nullptr;
    cudaStream_t cs = nullptr, cs2 = nullptr;   // capture streams of the body and of IF bodies
    uint32_t *ctl = nullptr;
    md_status rebuild_if(const NbrArgs &na, int ncell_total);
};
md_status run_captured_call(const void *key, size_t key_bytes, const std::function<md_status(cudaStream_t)> &body,
                            cudaStream_t st);
md_status run_graph_loop(const void *key, size_t key_bytes, uint32_t *ctl, int niter,
                         const std::function<md_status(LoopBuilder &)> &body, cudaStream_t st);
// FIRE (fire.cu): one step's launches, and what the rules of a step used
// (recorded for the reverse pass of the FIRE adjoint).
struct FireStep {
    float dt, alpha, keep;
    int freeze;
};
struct FireCtx {
    PairArgs pa;
    NbrArgs na;
    uint32_t *ctl;
    void *state;
    Box box;
    int N, dim, kind, ncell;
    float4 *r, *v, *f;
    const float4 *rref;
    float hs2;
    md_fire_params prm;
    uint32_t *status;
};
md_status fire_params_ok(const md_fire_params *fp);
bool make_fire_ctx(const md_space *s, const md_pot *p, const md_fire_params *fp, float *d_r, float *d_v, float *d_f,
                   md_nbr *nb, void *d_state, uint32_t *d_status, FireCtx &c);
void enqueue_fire_init(void *state, const md_fire_params &fp, cudaStream_t st);
md_status enqueue_fire_step(const FireCtx &c, FireStep *rec, cudaStream_t cs, LoopBuilder *lb);
// 1 (default): FIRE and flocking loops run as graph loops; 0: host launches.
extern int g_loop_graphs;
void enqueue_rebuild_chain(const NbrArgs &a, int ncell_total, cudaStream_t st);
void enqueue_cell_binning(const NbrArgs &a, int ncell_total, cudaStream_t st);
// Device loop counters: step 0 of nsteps (energy series index).
void enqueue_loop_init(uint32_t *ctl, uint32_t nsteps, cudaStream_t st);
void enqueue_check_disp(const md_space *s, const float *d_r, const md_nbr *nb, cudaStream_t st);

bool make_pair_args(const md_space *s, const md_pot *p, const float *d_r, const md_nbr *nb, float *d_f,
                    PairArgs &a);
void enqueue_pair(const PairArgs &a, int dim, int pot, int kick, cudaStream_t st);
// Force evaluation for any supported potential (pair kernels or SW).
void enqueue_forces(const PairArgs &a, int dim, int pot, int kick, cudaStream_t st);
void enqueue_sw(const PairArgs &a, int kick, cudaStream_t st);
constexpr int SW_LIST_SLOTS = 32;   // partners inside a*sigma kept per atom (more: overflow)
constexpr int BP_LIST_SLOTS = 48;   // partners inside R_c kept per atom by the learned potential
size_t sw_lists_bytes(int N);       // partner-list scratch of N atoms (tb_layout)
void enqueue_bp_step(const PairArgs &a, int kick, cudaStream_t st);
void enqueue_gnn_step(const PairArgs &a, int kick, cudaStream_t st);
bool gnn_model_ok(const md_gnn_model *m, const md_nbr *nb);
int bp_variant();
int gnn_variant();
int pair_blocks(int N, int tpp);
// Tile engine (tiles.cu): md_integrate_nve for LJ / soft spheres in 3-D on
// plans with MD_NBR_TILES.
bool tiles_enabled(const md_space *s, const md_nbr *nb, const md_pot *p);
bool tiles_plan_ok(const md_space *s, const md_nbr *nb);
md_status run_tiled_nve(const md_space *s, const md_pot *p, float *d_r, float *d_v, float *d_f, float mass, float dt,
                        int nsteps, md_nbr *nb, double *d_PE, double *d_KE, int use_graph, uint32_t *d_status,
                        cudaStream_t st);
// r += eta F (unwrapped) with the displacement check (gradient descent step)
void enqueue_gd_step(const md_space *s, float *d_r, const float *d_f, const md_nbr *nb, float eta, cudaStream_t st);

}  // namespace jmd


