/*
 * jmd.h -- C ABI of libjmd, the B300 (sm_103a) molecular-dynamics hot path.
 *
 * The calls follow the problem statement of "JAX, M.D.: A Framework for
 * Differentiable Physics" (Schoenholz & Cubuk, arXiv:1912.04232):
 *   periodic spaces                         Sec. 3.2.1
 *   pair interactions U = 1/2 sum u(r_ij)   Sec. 3.2.2
 *   cell lists and neighbor lists           Sec. 3.2.3
 *   NVE / NVT / minimisation                Sec. 3.3.1
 *   LJ, soft-sphere, Stillinger-Weber       Sec. 3.3.2
 *   neural-network potentials               Sec. 3.2.4, 4.1
 *   differentiating a minimisation          Sec. 4.2, App. A
 *
 * Conventions (every call):
 *   - Every call returns md_status.  Argument errors found on the host are
 *     returned synchronously and nothing is enqueued.  Errors that only the
 *     device can see (neighbor overflow, non-finite values, bounds, timeouts)
 *     are OR-ed into a caller-provided device word `uint32_t* d_status`; read
 *     it with md_status_poll().
 *   - All device arrays are owned by the caller.  The library never
 *     allocates or frees device memory.  Scratch comes from a caller buffer
 *     whose size the matching *_plan call reports.
 *   - Positions, velocities and forces are float[N][4] (16-byte aligned):
 *       positions  (x, y, z, w): w = particle diameter for soft spheres,
 *                   0 otherwise; z = 0 in 2-D;
 *       velocities (vx, vy, vz, 0);
 *       forces     (fx, fy, fz, e_i) where e_i is the per-particle energy,
 *                   so that sum_i e_i = U.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     is asynchronous on that stream unless stated otherwise.
 */
#ifndef JMD_H
#define JMD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define JMD_API __attribute__((visibility("default")))
#else
#define JMD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *md_stream_t; /* == cudaStream_t */

typedef enum {
    MD_OK = 0,
    MD_ERR_INVALID = 1,        /* bad argument (host) */
    MD_ERR_BOX_TOO_SMALL = 2,  /* box edge < 2 * interaction range: minimum image invalid */
    MD_ERR_NBR_OVERFLOW = 4,   /* a neighbor row needed more than `cap` slots (device) */
    MD_ERR_NONFINITE = 8,      /* a NaN / Inf reached a reduction (device) */
    MD_ERR_TIMEOUT = 16,       /* a bounded device wait ran out (device) */
    MD_ERR_BOUNDS = 32,        /* an index failed a bounds check (device) */
    MD_ERR_CUDA = 64           /* a CUDA runtime call failed (host) */
} md_status;

/* ------------------------------------------------------------------------ */
/* Periodic space (Sec. 3.2.1): the box [0,L_x) x [0,L_y) (x [0,L_z)) with   */
/* r ~ r + n L.  The displacement of a from b is the nearest-image vector    */
/*   t = a - b;  d = t - L * rint(t * Linv)                                  */
/* and the shift r + dr is wrapped back as r - L * floor(r * Linv).          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dim;          /* 2 or 3 */
    float L[3];       /* box edges in FP32 (unused axes = 1) */
    float Linv[3];    /* 1/L evaluated in FP64, rounded to FP32 */
    double L64[3];    /* box edges as given */
} md_space;

/* box: double[dim].  Fails with MD_ERR_INVALID for dim not in {2,3} or a
 * non-positive edge. */
JMD_API md_status md_space_periodic(int dim, const double *box, md_space *out);

/* ------------------------------------------------------------------------ */
/* Neighbor list (Sec. 3.2.3): for every i, the j != i with r_ij < r_list,   */
/* r_list = r_cut + skin, found through a cell list with cells of side       */
/* >= r_list.  Rows are padded with N; cnt[i] is the true count even when it */
/* exceeds cap (then MD_ERR_NBR_OVERFLOW is raised and the row truncated).   */
/* Row order is deterministic: grouped by stencil cell in a fixed order and  */
/* ascending inside each cell (fully ascending for cells whose stencil holds */
/* more than 1024 particles).  Membership is decided in FP32 as              */
/*   r2 = (dx*dx + dy*dy) + dz*dz < fl32(r_list)^2                           */
/* with every operation rounded separately (no FMA).                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dim, N, cap;
    int ncell[3];          /* cells per axis (>= 1; stencil deduplicated below 3) */
    int ncell_total;
    float r_cut, skin;
    float r_list;          /* fl32(r_cut + skin) */
    float r_list2;         /* fl32(r_list * r_list) */
    float half_skin2;      /* fl32((skin/2)^2): rebuild threshold on displacement^2 */
    float cell_scale[3];   /* ncell / L */
    size_t ws_bytes;       /* scratch needed by this plan */
    /* caller-owned device memory, bound with md_nbr_bind: */
    int32_t *nbr;          /* [N][cap] */
    int32_t *cnt;          /* [N] */
    float *rref;           /* [N][4] positions at the last build */
    void *ws;              /* ws_bytes of scratch (cells, sorted copy, control words, reduction partials) */
    int flags;             /* MD_NBR_* bits (md_nbr_set_flags, before md_nbr_bind), else 0 */
} md_nbr;

/* Canonical mode: every build also sorts each row ascending, and force
 * kernels on this list sum each particle's pairs one thread at a time in
 * row order.  A particle's force is then a function of the positions alone,
 * independent of when the list was last rebuilt, which makes minimisation
 * trajectories reproducible bit for bit from any checkpoint (the adjoint's
 * recomputation relies on it).  Slower; meant for small systems. */
#define MD_NBR_CANONICAL 1

/* Local rows: every build also writes, for each row entry, the entry's index
 * into the region of the particle's cell block as a 16-bit row in the
 * workspace.  Cells are grouped two per axis into blocks; a block's region is
 * the block grown by one cell on each side (periodic), its cells taken in
 * (z, y, x) order and their members in ascending particle order.  Pair
 * forces (Lennard-Jones, soft sphere) then run one CTA per block that stages
 * the region's positions in shared memory and gathers from there; the
 * forces are bitwise those of the int32 rows.  Blocks whose region holds
 * more than 2048 particles, or a cell whose stencil holds more than 1024,
 * and grids with fewer than 4 cells on an axis use the int32 rows.  An
 * opt-in: on B300 the int32-row gather kernel measured faster.  Not
 * combinable with MD_NBR_CANONICAL. */
#define MD_NBR_LOCAL_ROWS 2

/* Tiles: the workspace also holds a second, tiled copy of the system for
 * the velocity-Verlet loop of Lennard-Jones and soft-sphere particles in 3-D
 * (md_integrate_nve), which then runs on it.  Every rebuild (Sec. 3.2.3)
 * puts the particles in memory in the order of a grid of half-size cells
 * (side >= r_list / 2, twice the list's cells per axis, members of a
 * half-cell by ascending caller index), and writes each particle's row as
 * 16-bit indices into the positions of its tile's region.  A tile is a
 * block of tx x ty x tz half-cells (tx <= 2, ty, tz <= 8, chosen per plan,
 * md_tiles_info); its region is the tile grown by two half-cells on each
 * side (periodic), its half-cells in (z, y, x) order.  One CTA per tile stages the region's positions in shared memory
 * with bulk (TMA) copies and evaluates forces, the closing half-kick, the
 * next kick-drift and the displacement check from there.  The region's
 * copies from across the box are staged at their periodic image, so a
 * partner's nearest-image vector is the plain difference; between rebuilds
 * positions are not wrapped, so those images stay valid, and they are
 * wrapped at every rebuild and on return.  Membership is decided on those
 * staged positions (r^2 with FMAs, strict < r_list^2), so the pair sets
 * equal the int32 rows' except for pairs within an ulp of r_list; the
 * step's cutoff test takes the same form.  On return md_integrate_nve
 * writes r, v, f, the int32 rows, counts and build positions back in the
 * caller's order.
 * Needs dim = 3, at least 3 cells on every axis, r_cut > skin and cap a
 * multiple of 8; a region
 * holds at most about 1.25x its mean count plus 128 particles (denser
 * regions raise MD_ERR_NBR_OVERFLOW).  Not combinable with
 * MD_NBR_CANONICAL or MD_NBR_LOCAL_ROWS. */
#define MD_NBR_TILES 4

/* Plan a neighbor list for N particles in space s.  Fails with
 * MD_ERR_BOX_TOO_SMALL if any used box edge is < 2 r_list, MD_ERR_INVALID
 * for N < 1, cap < 1, r_cut <= 0 or skin < 0.  Fills out (pointers NULL). */
JMD_API md_status md_nbr_plan(const md_space *s, int N, float r_cut, float skin, int cap, md_nbr *out);

/* Set the MD_NBR_* bits of a plan and update its ws_bytes (local rows need
 * N*cap*2 more bytes, tiles about 120 + 2*cap bytes per particle).  Call
 * before md_nbr_bind; MD_ERR_INVALID for unknown bits, for combinations
 * the flags exclude, and for MD_NBR_TILES on a plan that cannot use it. */
JMD_API md_status md_nbr_set_flags(md_nbr *nb, int flags);

/* Attach caller memory: d_nbr [N*cap] int32, d_cnt [N] int32, d_rref [N*4]
 * float (16-byte aligned), d_ws [ws_bytes] (256-byte aligned).  Zeroes the
 * control words and the cell histogram of d_ws on `stream`. */
JMD_API md_status md_nbr_bind(md_nbr *nb, int32_t *d_nbr, int32_t *d_cnt, float *d_rref, void *d_ws,
                              md_stream_t stream);

/* Unconditional rebuild from positions d_r [N][4]. */
JMD_API md_status md_neighbor_list_build(const md_space *s, const float *d_r, md_nbr *nb, uint32_t *d_status,
                                         md_stream_t stream);

/* Rebuild only if some particle moved more than skin/2 from its position at
 * the last build (minimum image; the check runs on the device, the host
 * does not wait). */
JMD_API md_status md_neighbor_list_update(const md_space *s, const float *d_r, md_nbr *nb, uint32_t *d_status,
                                          md_stream_t stream);

/* Neighbor-list build that allocates nothing and needs no workspace.
 * The paper has no counterpart; this serves callers that cannot give the
 * library device memory beyond their own inputs and outputs (a host that
 * passes only its particle buffers through a plugin interface, or a loop
 * that must not pay for cudaMalloc).  It runs the same kernels as
 * md_neighbor_list_build and writes the same rows to d_nbr [N][cap] and
 * counts to d_cnt [N]; the scratch (cells, sorted copy, control words,
 * build positions) comes from a fixed pool of md_noalloc_scratch_bytes()
 * bytes inside the library, held by every GPU that loads it until exit.
 *   - Returns MD_ERR_INVALID when N and the cell grid need more scratch
 *     than the pool holds, besides the md_nbr_plan errors.  The need is
 *     about 68 bytes per particle plus 8 per cell (the md_nbr_plan
 *     workspace rounded up to 256 bytes, plus 16 bytes per particle of
 *     build positions): 61,248 particles fit for LJ at density 0.84 with
 *     r_list 2.8 (box 42.06, 15^3 cells), 61,249 do not.  It calls no
 *     allocating routine.
 *   - Outside stream capture every call looks up the pool's device address
 *     (cudaGetSymbolAddress) with the current device; a captured call reuses
 *     the address of the last uncaptured one on that device.  Make one
 *     uncaptured call per device before the first capture, and again after
 *     a cudaDeviceReset.
 *   - All calls on a device share that device's pool, which keeps the last
 *     call's contents (the parts that must start at zero are cleared by
 *     every call); calls that can overlap on the same GPU, for example on
 *     two streams, race on it. */
JMD_API md_status md_neighbor_list_build_noalloc(const md_space *s, const float *d_r, int N, float r_cut, float skin,
                                                 int cap, int32_t *d_nbr, int32_t *d_cnt, uint32_t *d_status,
                                                 md_stream_t stream);

/* Spatial sort (data layout for the gather kernels; the paper has no
 * counterpart: its particle order is whatever the caller supplies).  The pair
 * kernels gather every neighbor's position; how often a gathered cache line
 * is reused depends on whether particles close in space are close in memory.
 * A lattice start has that order, diffusion destroys it (random order makes
 * the LJ force kernel at N = 256,000 1.7x slower).  This call renumbers the
 * particles: the cells of the plan's grid in Z-order (Morton) of their
 * coordinates, each cell's members in ascending old index.  The permutation
 * is a deterministic function of the positions and the grid.
 *   d_r: float[N][4] positions (with w), permuted in place.
 *   d_v: float[N][4] velocities permuted in place, or NULL.
 *   d_perm: int32[N] out, d_perm[new] = old index.  Any other per-particle
 *     array (forces, species) must be permuted by the caller with it, or
 *     recomputed.
 *   d_scratch: md_sort_scratch_bytes(nb) bytes of caller device memory,
 *     256-byte aligned.
 * The call rebuilds the list for the new order (as md_neighbor_list_build).
 * A particle's row then holds the same partners in the same order, so its
 * force keeps its bits (later rebuilds order each cell by the new indices,
 * so trajectories agree to the rounding of reordered sums).  MD_ERR_INVALID for null pointers, a plan that is
 * not bound, misaligned or too small scratch, or a grid with more than 2^24
 * Z-order keys (more than 256 cells on an axis in 3-D, 4,096 in 2-D). */
JMD_API md_status md_sort_particles(const md_space *s, md_nbr *nb, float *d_r, float *d_v, int32_t *d_perm,
                                    void *d_scratch, size_t scratch_bytes, uint32_t *d_status, md_stream_t stream);

/* Scratch bytes md_sort_particles needs for this plan (0 if the grid is too
 * large to sort). */
JMD_API size_t md_sort_scratch_bytes(const md_nbr *nb);

/* Size in bytes of the pool used by md_neighbor_list_build_noalloc. */
JMD_API size_t md_noalloc_scratch_bytes(void);

/* Synchronous on `stream`: builds done since bind, largest row count seen
 * by any build since bind. */
JMD_API md_status md_nbr_stats(const md_nbr *nb, int64_t *builds, int32_t *max_count, md_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Energy functions (Sec. 3.3.2) summed over the neighbor list (smap.neighbors,
 * Sec. 3.2.2): U = 1/2 sum_{i != j} u(r_ij), F = -grad U.                   */
/* ------------------------------------------------------------------------ */
typedef enum { MD_LJ = 0, MD_SOFT_SPHERE = 1, MD_SW = 2, MD_BP = 3, MD_GNN = 4 } md_potential;

typedef struct {
    md_potential kind;
    /* MD_LJ: u = 4 eps [(sigma/r)^12 - (sigma/r)^6] - e_shift for r < r_cut
     * (the r < r_cut test in FP32 as for the neighbor list); forces unshifted. */
    float eps, sigma, r_cut, e_shift;
    /* MD_SOFT_SPHERE: u = (eps/alpha) (1 - r/s_ij)^alpha for r < s_ij,
     * s_ij = (w_i + w_j)/2 from the position w column. */
    float alpha;
    /* MD_SW: {eps, sigma, a, lambda, gamma, A, B, p, q, cos0}; cutoff a*sigma. */
    float sw[10];
    /* MD_BP: pointer to an md_bp_model; MD_GNN: pointer to an md_gnn_model.
     * MD_SW: NULL, or device scratch of md_sw_lists_bytes(N) bytes (256-byte
     * aligned, caller-owned, contents scratch) for the list's N atoms.  With
     * it each evaluation first stores every atom's partners inside a*sigma
     * (at most 32; more raise MD_ERR_NBR_OVERFLOW) and the triplets centred
     * on a neighbor visit only that neighbor's stored partners; without it
     * one kernel tests the neighbors' whole rows.  Both give the same terms;
     * their FP32 sums may differ in the last bits (another summation order). */
    const void *model;
} md_pot;

/* Bytes of the MD_SW partner-list scratch for N atoms (0 if N < 1). */
JMD_API size_t md_sw_lists_bytes(int N);

/* Learned potential (MD_BP, Sec. 3.2.4 and 4.1): Behler-Parrinello
 * symmetry functions (8 radial, 8 angular; cutoff 3.77 A) feeding a per-atom
 * network 16 -> 64 -> 64 -> 1 with SiLU.  All pointers are device memory
 * owned by the caller. */
typedef struct {
    const float *params;  /* [5313] FP32: W1 [64][16], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 */
    const float *norm;    /* [32] FP32: descriptor mean [16] then standard deviation [16] */
    float *G;             /* [N][16] scratch: descriptors */
    float *dEdG;          /* [N][16] scratch: network input gradient */
    float *Ei;            /* [N] scratch: per-atom energies */
    int sys_n;            /* 0, or atoms per system for concatenated equal-size systems */
    void *lists;          /* NULL, or scratch of md_bp_lists_bytes(N) bytes (256-byte aligned): the
                             descriptor kernel then stores every atom's partners inside R_c (at most
                             48; more raise MD_ERR_NBR_OVERFLOW) and the force gather visits only the
                             neighbors' stored partners for the triplets centred on them (the same
                             terms; FP32 sums may differ in the last bits) */
} md_bp_model;

/* Bytes of the md_bp_model partner-list scratch for N atoms (0 if N < 1). */
JMD_API size_t md_bp_lists_bytes(int N);

/* Graph-network potential (MD_GNN; Sec. 3.2.4: GraphNet blocks as in the
 * glass network of Bapst et al.; Sec. 4.1: trained on energies and forces,
 * not rotation invariant).  The paper prints no architecture; this one is
 * encode - process - decode with hidden width H and T message-passing steps
 * on the directed edges (i <- j), r_ij < r_cut, of a 3-D neighbor list:
 *   e_ij = silu(W_enc x_ij + b_enc),  x_ij = (R_j - R_i) / r_cut;  v_i = u
 *   step t = 1..T:  e_ij = silu(A_e e_ij + A_r v_i + A_s v_j + a)
 *                   m_i  = sum_j s(r_ij) e_ij,  s(r) = (cos(pi r / r_cut) + 1) / 2
 *                   v_i  = silu(B_v v_i + B_m m_i + b)
 *   E_i = w . silu(D v_i + d) + c,  E = sum_i E_i,  F = -dE/dR  (FP32).
 * params (device, md_gnn_param_count(H, T) floats, row-major blocks):
 *   W_enc [H][3], b_enc [H], u [H],
 *   T x { A [H][3H] (columns A_e | A_r | A_s), a [H], B [H][2H] (B_v | B_m), b [H] },
 *   D [H][H], d [H], w [H], c.
 * ws: device scratch of md_gnn_workspace_bytes(N, cap, H, T) bytes for the
 * list the model is evaluated on (caller-owned; contents are scratch).
 * Needs H in {32, 64}, 1 <= T <= 4, r_cut <= the list's r_list, cap <= 64
 * and a symmetric list (every pair in both rows; a missing reverse entry
 * raises MD_ERR_NBR_OVERFLOW).  md_energy_forces writes F and E_i to
 * d_f [N][4]. */
typedef struct {
    const float *params;
    int H, T;
    float r_cut;
    void *ws;
    size_t ws_bytes;
    int sys_n;            /* 0, or atoms per system for concatenated equal-size systems (rows local to each) */
} md_gnn_model;

/* Parameter count 5H + T (5H^2 + 2H) + H^2 + 2H + 1; 0 for unsupported H, T. */
JMD_API size_t md_gnn_param_count(int H, int T);
/* 1: the products of md_energy_forces with MD_GNN run on the tensor cores
 * (tcgen05, BF16 operands, FP32 accumulation; H = 64 only, other widths
 * keep the FP32 kernels), the edges compacted in receiver order; 0
 * (default): FP32 CUDA-core kernels.  MD_ERR_INVALID for other values. */
JMD_API md_status md_gnn_set_tensor_cores(int on);
/* Atoms per warp of the network kernels (1, 2, 4 or 8; default 4): more
 * atoms share each weight read, fewer warps hide latency.  The forces do
 * not depend on it.  MD_ERR_INVALID for other values. */
JMD_API md_status md_gnn_set_group(int G);
/* Workspace bytes for N atoms and row capacity cap; 0 if unsupported. */
JMD_API size_t md_gnn_workspace_bytes(int N, int cap, int H, int T);

/* Training (Sec. 4.1: the network is fitted to energies and forces).
 * Gradient with respect to the parameters of
 *     J = sum_i c_E,i E_i - sum_k u_k . dE/dR_k
 * which, with c_E = dL/dE_i and u = dL/dF_k (md_bp_loss_prep: d_cE [N],
 * d_dF [N][4]), is the gradient of the energy + force loss L.  The force
 * term needs second derivatives: the network runs forward carrying the
 * tangent along u, then one reverse sweep goes through values and tangents;
 * weight gradients are summed over edges and atoms in a fixed order (FP64
 * across row batches).  FP32 kernels; H = 64 only.  d_r, nb: the atoms
 * (N = nb->N), all in the box s; with m->sys_n > 0 they are systems of
 * sys_n atoms whose rows are local to each system.  m: the model (its
 * workspace for this N and cap is used as scratch too).  d_scratch:
 * md_gnn_train_scratch_bytes(N, cap, H, T) bytes, 256-byte aligned.
 * d_grad: md_gnn_param_count(H, T) floats, overwritten. */
JMD_API size_t md_gnn_train_scratch_bytes(int N, int cap, int H, int T);
JMD_API md_status md_gnn_train_grad(const md_space *s, const float *d_r, const md_nbr *nb, const md_gnn_model *m,
                                    const float *d_cE, const float *d_dF, void *d_scratch, size_t scratch_bytes,
                                    float *d_grad, uint32_t *d_status, md_stream_t stream);

/* Forces and per-particle energies into d_f [N][4]; if d_E != NULL the FP64
 * total energy sum_i e_i is written to *d_E (device).  Needs a built list
 * with r_list >= the potential's range and positions inside the box [0, L)
 * (as the integrators keep them; md_minimize accepts unwrapped ones). */
JMD_API md_status md_energy_forces(const md_space *s, const md_pot *p, const float *d_r, const md_nbr *nb,
                                   float *d_f, double *d_E, uint32_t *d_status, md_stream_t stream);

/* Threads per particle of the pair-force kernels (4, 8, 16 or 32): the
 * group that gathers one row.  A tuning knob; results are identical up to
 * FP32 summation order. */
JMD_API md_status md_set_pair_tpp(int tpp);

/* Pair-kernel variant (LJ and soft-sphere gather kernels).  Bit 0: read the
 * neighbor rows past L1 (default 1, measured faster on B300) or through it.
 * Bit 1: check every row entry against [0, N) before its position is
 * gathered; an entry outside is skipped and ORs MD_ERR_BOUNDS into the status
 * word (diagnosing a corrupted list; without it such an entry reads outside
 * the positions).  On valid lists every variant gives the same bits.  Other
 * values: MD_ERR_INVALID. */
JMD_API md_status md_set_pair_options(int opt);

/* NVE with Lennard-Jones or soft-sphere forces on int32 rows: 1 (default)
 * fuses each step's kick-drift into the previous step's force kernel, with
 * the positions alternating between d_r and a workspace buffer (the final
 * positions are copied back to d_r); 0 runs the separate kick-drift kernel.
 * Both give the same bits.  MD_ERR_INVALID for other values. */
JMD_API md_status md_set_nve_fusion(int on);

/* Gradient descent (md_minimize), FIRE (md_minimize_fire) and flocking
 * (md_flock_run) loops: 1 (default) run each call as one CUDA graph with a
 * device-controlled loop and the rebuild chain under a conditional node.
 * The adjoints (md_minimize_adjoint, md_minimize_fire_adjoint): 1 captures
 * each call's fixed launch sequence once per argument set and replays it as
 * one graph (at most 32 kept; evicting the oldest waits for the device to
 * be idle).  0 launches every kernel from the host.  Both give the same
 * bits.  MD_ERR_INVALID for other values. */
JMD_API md_status md_set_loop_graphs(int on);

/* ------------------------------------------------------------------------ */
/* Dynamics (Sec. 3.3.1).                                                   */
/* ------------------------------------------------------------------------ */
/* Nose-Hoover chain NVT (Sec. 3.3.1, Nose-Hoover constant temperature;
 * Martyna, Klein, Tuckerman 1992).  Each step is the symmetric splitting
 * chain(dt/2) . kick(dt/2) . drift(dt) . kick(dt/2) . chain(dt/2), the chain
 * half-step being the sweep of Martyna, Tuckerman, Tobias, Klein (1996)
 * with one sub-step; g = dim N, Q_1 = g kT tau^2, Q_k = kT tau^2.  Any
 * potential of md_energy_forces.  d_therm: md_nhc_state_doubles(M) device
 * doubles, caller-owned: chain positions xi[M], velocities w[M], masses and
 * constants; reset = 1 zeroes xi and w, reset = 0 continues.  d_PE, d_KE,
 * d_H (nsteps doubles each, may be NULL): potential, kinetic and conserved
 * extended energy H' = K + U + sum Q_k w_k^2/2 + g kT xi_1 + kT sum_{k>1} xi_k
 * after each step.  1 <= M <= 8, kT > 0, tau > 0, else MD_ERR_INVALID.
 * Positions stay inside [0, L). */
JMD_API size_t md_nhc_state_doubles(int M);
JMD_API md_status md_integrate_nhc(const md_space *s, const md_pot *p, float *d_r, float *d_v, float *d_f, float mass,
                                   float dt, float kT, float tau, int M, int nsteps, md_nbr *nb, double *d_therm,
                                   int reset, double *d_PE, double *d_KE, double *d_H, int use_graph,
                                   uint32_t *d_status, md_stream_t stream);

/* nsteps of velocity-Verlet NVE.  On entry d_f must hold the forces at d_r
 * (md_energy_forces) and nb a list built for d_r (with MD_NBR_TILES the run
 * imports d_r and builds its own rows; see that flag).  Each step:
 *   v += dt/2 F/m;  r = wrap(r + dt v);  rebuild the list if needed;
 *   F = F(r);       v += dt/2 F/m;
 * mass is in energy*time^2/length^2.  d_PE / d_KE (nsteps doubles each, may
 * be NULL) receive the FP64 potential and kinetic energy after each step.
 * use_graph != 0 runs the whole loop as one CUDA graph launch with device-
 * side loop control (captured once per argument set and cached; the first
 * call with a new argument set must not happen during a stream capture). */
JMD_API md_status md_integrate_nve(const md_space *s, const md_pot *p, float *d_r, float *d_v, float *d_f,
                                   float mass, float dt, int nsteps, md_nbr *nb, double *d_PE, double *d_KE,
                                   int use_graph, uint32_t *d_status, md_stream_t stream);

/* The tile engine (MD_NBR_TILES) as separate calls, for callers that
 * evaluate forces on it without integrating (and for timing its force
 * kernel alone).  The tiled copy lives in nb's workspace.
 *   md_tiles_import: copies d_r, d_v (may be NULL: zero) and d_f (may be
 *     NULL) into the tiled order and builds its rows from d_r (wrapped).
 *   md_tiles_forces: Lennard-Jones or soft-sphere forces and per-particle
 *     energies at the tiled positions into the tiled force array; d_E (one
 *     double, may be NULL) receives the FP64 potential energy.  One launch
 *     of the tile force kernel.
 *   md_tiles_export: writes positions (wrapped), velocities and forces back
 *     to d_r, d_v, d_f in the caller's order (any may be NULL) and, with
 *     rows != 0, the tiled rows as the caller's int32 rows, counts and build
 *     positions (nb->nbr, cnt, rref), so that nb is a valid list for the
 *     exported positions.
 * MD_ERR_INVALID if nb lacks MD_NBR_TILES or is not bound, or for other
 * potentials. */
JMD_API md_status md_tiles_import(const md_space *s, const float *d_r, const float *d_v, const float *d_f, md_nbr *nb,
                                  uint32_t *d_status, md_stream_t stream);
JMD_API md_status md_tiles_forces(const md_space *s, const md_pot *p, md_nbr *nb, double *d_E, uint32_t *d_status,
                                  md_stream_t stream);
JMD_API md_status md_tiles_export(const md_space *s, md_nbr *nb, float *d_r, float *d_v, float *d_f, int rows,
                                  md_stream_t stream);

/* nsteps velocity-Verlet steps on the tiled copy with its rows held fixed
 * (no rebuild): the opening half-kick and drift, then one launch of the
 * fused step kernel per step (forces, closing half-kick, next kick-drift,
 * displacement check).  Valid while no particle moves more than skin/2 from
 * its position at the last build (the rebuild flag is raised, not acted
 * on); md_integrate_nve is the call that rebuilds.  On return the tiled
 * copy holds r, v and F of the last step (md_tiles_export).  d_PE, d_KE as
 * in md_integrate_nve. */
JMD_API md_status md_tiles_steps(const md_space *s, const md_pot *p, md_nbr *nb, float mass, float dt, int nsteps,
                                 double *d_PE, double *d_KE, uint32_t *d_status, md_stream_t stream);

/* Geometry the tile engine chose for a plan: half-cells per axis (3), the
 * tile's extent along x, y and z (3), number of tiles, region capacity in
 * particles.  out: 8 ints.  MD_ERR_INVALID if the plan cannot use tiles. */
JMD_API md_status md_tiles_info(const md_space *s, const md_nbr *nb, int32_t *out);

/* Lanes per particle of the tile force kernel: 1, 4 or 8, or 0 (default)
 * to choose by tile size (1 for tiles of at least 128 particles, else 4). */
JMD_API md_status md_set_tile_tpp(int tpp);

/* nsteps of BAOAB Langevin dynamics at constant temperature (Sec. 3.3.1,
 * "Langevin ... simulations at constant temperature"), 3-D only:
 *   v += dt/2 F/m; r += dt/2 v; v = c1 v + c2 z; r += dt/2 v; F = F(r); v += dt/2 F/m
 * with c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT / m).  z are standard
 * normals from Philox4x32-10 with key `seed` and counter (i, step0 + k, 0, 0)
 * at step k, through Box-Muller on uniforms ((x >> 8) + 1) 2^-24.  Other
 * arguments and the graph behaviour as md_integrate_nve. */
JMD_API md_status md_integrate_langevin(const md_space *s, const md_pot *p, float *d_r, float *d_v, float *d_f,
                                        float mass, float dt, float gamma, float kT, uint64_t seed, uint32_t step0,
                                        int nsteps, md_nbr *nb, double *d_PE, double *d_KE, int use_graph,
                                        uint32_t *d_status, md_stream_t stream);

/* Minimisation (Sec. 3.3.1): kind 0 = gradient descent r <- r + step * F in
 * unwrapped coordinates (the list bins wrapped copies).  d_E (nsteps+1
 * doubles, may be NULL) receives U before every step and after the last;
 * d_f holds F at the final positions on return. */
JMD_API md_status md_minimize(const md_space *s, const md_pot *p, int kind, float step, int nsteps, float *d_r,
                              float *d_f, md_nbr *nb, double *d_E, uint32_t *d_status, md_stream_t stream);

/* FIRE (Sec. 3.3.1 minimisers; Bitzek et al., PRL 97, 170201 (2006)), unit
 * mass, unwrapped coordinates as in md_minimize.  Each step: velocity-Verlet
 * MD step with the current dt; P = F.v, |v|, |F| over all degrees of
 * freedom (FP64 sums); v = (1 - alpha) v + alpha |v| F/|F|; if P > 0 the
 * count of consecutive P > 0 steps grows and, once above n_min, dt =
 * min(dt f_inc, dt_max) and alpha *= f_alpha; if P <= 0, dt *= f_dec, v = 0,
 * alpha = alpha_start and the count restarts. */
typedef struct {
    float dt_start, dt_max, f_inc, f_dec, alpha_start, f_alpha;
    int n_min;
} md_fire_params;

/* Bytes of the device FIRE state (dt, alpha, count, reduction partials). */
JMD_API size_t md_fire_state_bytes(void);

/* nsteps of FIRE on d_r [N][4] (LJ or soft sphere; nb built for d_r).
 * restart = 1 starts from rest (d_v zeroed, state reset); restart = 0
 * continues from d_v [N][4] and d_state (md_fire_state_bytes, 256-byte
 * aligned, from an earlier restart).  d_E (nsteps+1 doubles, may be NULL)
 * receives U before every step and after the last; d_f holds F at the final
 * positions.  MD_ERR_INVALID for parameters outside dt_start > 0, dt_max >=
 * dt_start, f_inc >= 1, 0 < f_dec < 1, 0 <= alpha_start < 1,
 * 0 < f_alpha <= 1, n_min >= 0. */
JMD_API md_status md_minimize_fire(const md_space *s, const md_pot *p, const md_fire_params *fp, int nsteps,
                                   float *d_r, float *d_v, float *d_f, md_nbr *nb, void *d_state, int restart,
                                   double *d_E, uint32_t *d_status, md_stream_t stream);

/* Copies (dt, alpha, count of consecutive P > 0 steps) of a FIRE state to
 * the host (synchronises the stream). */
JMD_API md_status md_fire_state_read(const void *d_state, double *out3, md_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Flocking energy model (Sec. 4.3 and its appendix), 2-D periodic square.   */
/* ------------------------------------------------------------------------ */
/* Boids: positions R_i, headings theta_i, N_i = (cos, sin) theta_i.  With
 * rho(r; Rc) = (1 - r/Rc)^alpha / alpha below Rc and each unordered pair once:
 *   E_align    = sum J_align rho(r_ij; R_align) (1 - N_i.N_j)^2
 *   E_avoid    = sum J_avoid rho(r_ij; R_avoid)
 *   E_cohesion = sum_i J_cohesion/2 (1 - u_i.N_i)^2, u_i the unit vector
 *                towards the mean offset of the boids within R_cohesion
 *   E_obstacle = sum_i sum_o J_obstacle rho(|R_o - R_i|; D_o) (1 + N_i.w_io)^2,
 *                w_io the unit vector from boid i to disk obstacle o
 * Alignment and cohesion turn the boids only (no gradient through the
 * displacements).  Forward Euler: R_i += dt (speed N_i - dE/dR_i) (wrapped),
 * theta_i -= dt dE/dtheta_i.
 * Predators (position, heading), a two-player game: the boids add
 *   E_flee     = sum_i sum_p J_flee rho(|R_p - R_i|; R_flee) (1 + N_i.w_ip)^2
 * (the obstacle form), the predators minimise their own energy, the
 * cohesion form towards the boids within R_chase (heading only) plus the
 * obstacle terms, with forward-Euler steps at predator_speed.  The paper
 * lets predators sprint without defining it: here they swim at
 * predator_speed * sprint_factor in the steps s (counted from 0 in each
 * md_flock_run call) with s mod sprint_period < sprint_steps. */
typedef struct {
    float J_align, R_align, J_avoid, R_avoid, J_cohesion, R_cohesion, J_obstacle, alpha, speed;
    float J_flee, R_flee, J_chase, R_chase, predator_speed;   /* predators */
    int sprint_period, sprint_steps;                         /* sprints; period 0: none */
    float sprint_factor;
} md_flock_params;

/* nsteps of the flocking dynamics.  d_b [N][4]: (x, y, -, -) in, (x, y,
 * cos theta, sin theta) out; d_theta [N] headings in/out; d_b_alt [N][4]
 * scratch; d_obs [n_obs][3] (x, y, radius) device; d_pred [n_pred][4]
 * predators (x, y, theta, -) in/out (w: the predator's energy of the last
 * state), d_pred_alt [n_pred][4] scratch.  nb: a 2-D list built for d_b with
 * r_cut >= max(R_align, R_avoid, R_cohesion); rebuilt as the boids move.
 * d_E (nsteps doubles, may be NULL): the total energy (boids' and
 * predators') before each step. */
JMD_API md_status md_flock_run(const md_space *s, const md_flock_params *prm, const float *d_obs, int n_obs,
                               float *d_pred, float *d_pred_alt, int n_pred, float *d_b, float *d_theta,
                               float *d_b_alt, float dt, int nsteps, md_nbr *nb, double *d_E, uint32_t *d_status,
                               md_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Learned potential: the pieces of a forward/backward and a training step   */
/* (Sec. 4.1: energy + force loss).  sys_n as in md_bp_model.                */
/* ------------------------------------------------------------------------ */
/* G [N][16] from positions (list with r_list >= 3.77 A). */
JMD_API md_status md_bp_descriptors(const md_space *s, const float *d_r, const md_nbr *nb, int sys_n, float *d_G,
                                    uint32_t *d_status, md_stream_t stream);

/* Per-atom network: E_i [N] and dE_i/dG_i [N][16] (FP32). */
JMD_API md_status md_bp_mlp_infer(const float *d_params, const float *d_norm, const float *d_G, int N, float *d_Ei,
                                  float *d_dEdG, md_stream_t stream);

/* The same network on the tensor cores: tcgen05 MMAs with BF16 operands and
 * FP32 accumulation in tensor memory, 128 atoms per tile (4 MMAs: two
 * forward layers, two backward products).  BF16 rounding of the inputs and
 * hidden activations makes it agree with md_bp_mlp_infer to about 1e-2
 * relative.  Device waits are bounded: MD_ERR_TIMEOUT in *d_status. */
JMD_API md_status md_bp_mlp_infer_tc(const float *d_params, const float *d_norm, const float *d_G, int N,
                                     float *d_Ei, float *d_dEdG, uint32_t *d_status, md_stream_t stream);

/* Which network kernel MD_BP force evaluations use: 1 = tensor cores (BF16),
 * 0 = FP32 CUDA cores (default). */
JMD_API md_status md_bp_set_tensor_cores(int on);

/* F_k = -sum_i dE_i/dG_i . dG_i/dr_k into d_f [N][4] (w = E_k when d_Ei is
 * given); optional FP64 total of d_Ei into *d_E. */
JMD_API md_status md_bp_forces(const md_space *s, const float *d_r, const md_nbr *nb, int sys_n,
                               const float *d_dEdG, const float *d_Ei, float *d_f, double *d_E, uint32_t *d_status,
                               md_stream_t stream);

/* V_i = sum_k dG_i/dr_k . dF_k (descriptor Jacobian applied to d_dF [N][4]). */
JMD_API md_status md_bp_jvp(const md_space *s, const float *d_r, const md_nbr *nb, int sys_n, const float *d_dF,
                            float *d_V, uint32_t *d_status, md_stream_t stream);

/* Scratch bytes of md_bp_mlp_train for N atoms. */
JMD_API size_t md_bp_train_scratch_size(int N);

/* Gradient of J = sum_i [c_E,i E_i - c_F dE_i/dG_i . V_i] with respect to the
 * packed parameters into d_grad [5313].  With c_E,i = 2 (E_s - E_ref,s) /
 * (S N^2) for atom i of snapshot s and V = the JVP of c_F-scaled force
 * errors this is the gradient of the energy + force loss. */
JMD_API md_status md_bp_mlp_train(const float *d_params, const float *d_norm, const float *d_G, const float *d_V,
                                  const float *d_cE, float cF, int N, void *d_scratch, float *d_grad,
                                  md_stream_t stream);

/* The same gradient on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation in tensor memory): per 128-atom tile the forward pass, its
 * tangent and the reverse pass as MMAs, and the sums over atoms as MMAs
 * with the atoms as K, accumulated across tiles; each CTA's partial
 * gradient is then added in CTA order in FP64 (deterministic).  BF16
 * rounding of the weights, inputs and per-atom factors keeps it within
 * about 1e-2 of md_bp_mlp_train (relative to the gradient's norm).
 * d_G, d_V and d_scratch (md_bp_train_scratch_size(N) bytes) 16-byte
 * aligned.  Device waits are bounded: MD_ERR_TIMEOUT in *d_status. */
JMD_API md_status md_bp_mlp_train_tc(const float *d_params, const float *d_norm, const float *d_G, const float *d_V,
                                     const float *d_cE, float cF, int N, void *d_scratch, float *d_grad,
                                     uint32_t *d_status, md_stream_t stream);

/* Loss of the energy + force fit (Sec. 4.1) over S snapshots of n atoms:
 *   loss = mean_s ((E_s - E_ref,s) / n)^2 + w_F mean (F - F_ref)^2
 * Writes c_E [S n] and dF [S n][4] (the force errors scaled by
 * 2 w_F / (3 n S), to feed md_bp_jvp and md_bp_mlp_train with c_F = 1) and
 * the per-snapshot loss terms d_loss [2 S] (energy, force). */
JMD_API md_status md_bp_loss_prep(const float *d_Ei, const float *d_F, const float *d_Fref, const double *d_Eref,
                                  int S, int n, float wF, float *d_cE, float *d_dF, double *d_loss,
                                  md_stream_t stream);

/* Column means then standard deviations of X [N][D] into d_out [2 D] (FP64
 * accumulation): the descriptor normalisation of the network. */
JMD_API md_status md_column_stats(const float *d_X, int N, int D, float *d_out, md_stream_t stream);

/* Adam (bias-corrected) on an FP32 vector; step counts from 1. */
JMD_API md_status md_adam_step(float *d_params, const float *d_grad, float *d_m, float *d_v, int n, float lr,
                               float beta1, float beta2, float eps, int step, md_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Differentiating through minimisation (Sec. 4.2, App. A): the final energy */
/* of T gradient-descent steps of a 2-D bidisperse soft-disk packing and its */
/* derivative with respect to the diameter D of the first nA disks (the rest */
/* have diameter dB).  The box is L(D) at packing fraction phi.              */
/* ------------------------------------------------------------------------ */
/* The packing's space: a square of edge
 *   L(D) = sqrt((nA pi D^2 / 4 + (N - nA) pi dB^2 / 4) / phi)
 * (FP64; out->L holds it rounded to FP32) and, if dLdD is not NULL,
 * dL/dD = pi nA D / (4 phi L).  MD_ERR_INVALID for N < 1, nA outside
 * [0, N] or non-positive D, dB, phi. */
JMD_API md_status md_packing_space(int N, int nA, double D, double dB, double phi, md_space *out, double *dLdD);

/* Workspace bytes for N particles, T steps, checkpoints every K steps:
 * (ceil(T/K) + K + 2) * N * 16. */
JMD_API size_t md_adjoint_workspace_size(int N, int T, int K);

/* r_0 = L s_0 (d_s0 [N][4] fractional coordinates), T steps of
 * r <- r + eta F(r) (soft spheres, p), E = U(r_T); hand-written reverse
 * mode with recomputation from checkpoints every K steps (K = ceil(sqrt T)
 * is the natural choice).  nb must be planned for this space with
 * r_cut >= max(D, dB), bound, and in MD_NBR_CANONICAL mode; the result is
 * then identical for every K.  s must be the packing's space
 * (md_packing_space(N, nA, D, dB, phi)); the library forms L(D) and dL/dD
 * itself, MD_ERR_INVALID if s is another box.  d_r [N][4] receives r_T
 * (w = diameter), d_f the forces at r_T; d_out[0] = E (FP64),
 * d_out[1] = dE/dD (FP64). */
JMD_API md_status md_minimize_adjoint(const md_space *s, const md_pot *p, md_nbr *nb, const float *d_s0, int nA,
                                      float D, float dB, double phi, float eta, int T, int K, float *d_r, float *d_f,
                                      void *d_ws, double *d_out, uint32_t *d_status, md_stream_t stream);

/* FIRE instead of gradient descent (Sec. 3.3.1 minimiser; Bitzek et al.,
 * PRL 97, 170201 (2006)): r_0 = L s_0 from rest, T FIRE steps with the
 * parameters fp, E = U(r_T) and dE/dD by hand-written reverse mode through
 * every step (velocity Verlet, the global norms of the mixing, the forces
 * via Hessian-vector products, the box and the diameters), with the time
 * steps, mixing factors and P > 0 decisions of the trajectory held fixed
 * (the map is piecewise smooth).  States (r, v and the FIRE scalars) are
 * kept every K steps and each segment is replayed bit for bit in the
 * reverse sweep; nb and s as for md_minimize_adjoint (canonical list, the
 * packing's space at phi), so the result is identical for every K.  d_ws: md_fire_adjoint_workspace_size(N, T, K)
 * bytes, 256-byte aligned.  d_r, d_v, d_f receive r_T, v_T, F(r_T);
 * d_out[0] = E, d_out[1] = dE/dD (FP64). */
JMD_API size_t md_fire_adjoint_workspace_size(int N, int T, int K);
JMD_API md_status md_minimize_fire_adjoint(const md_space *s, const md_pot *p, const md_fire_params *fp,
                                           md_nbr *nb, const float *d_s0, int nA, float D, float dB, double phi,
                                           int T, int K, float *d_r, float *d_v, float *d_f, void *d_ws,
                                           double *d_out, uint32_t *d_status, md_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batched replicas (the paper's vmap over independent systems, Sec. 4.2):   */
/* replicas of different size, box, density and potential (LJ or soft        */
/* spheres, 3-D) concatenated particle-wise and advanced by the same kernels */
/* -- one CUDA graph launch for a whole NVE run.                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int N;            /* particles */
    double L;         /* cubic box edge */
    int kind;         /* MD_LJ or MD_SOFT_SPHERE */
    float eps, sigma, r_cut, e_shift;   /* LJ (as md_pot); soft: eps, r_cut = max diameter */
    float alpha;      /* soft-sphere exponent */
    float skin, dt, mass;
    float cell_mult;  /* cell side >= cell_mult (r_cut + skin); values <= 1 mean 1 (the
                         smallest cells).  Larger cells mean fewer, fuller cells per
                         replica (a tuning knob, see md_batch_set_class_tpp); the rows
                         hold the same partners, in another order. */
} md_replica_desc;

typedef struct {
    int R, N, cap;        /* replicas, total particles, neighbor slots per row */
    int ncell_total;      /* cells of all replicas plus one end sentinel each */
    int tpp;              /* threads per particle of the force kernel (4, 8, 16) */
    size_t ws_bytes;      /* scratch the caller provides */
    int32_t *nbr;         /* [N][cap] rows with global particle indices */
    int32_t *cnt;         /* [N] */
    float *rref;          /* [N][4] */
    void *ws;             /* ws_bytes (256-byte aligned) */
    void *host;           /* library-owned host state; release with md_batch_free */
} md_batch;

/* Plan R replicas (reps[k] describes replica k; particles of replica k are
 * the next reps[k].N rows of the concatenated arrays).  Each replica's box
 * must hold twice its r_cut + skin (MD_ERR_BOX_TOO_SMALL otherwise). */
JMD_API md_status md_batch_plan(const md_replica_desc *reps, int R, int cap, md_batch *out);
JMD_API void md_batch_free(md_batch *bt);
/* Attach caller memory and upload the replica tables (synchronous). */
JMD_API md_status md_batch_bind(md_batch *bt, int32_t *d_nbr, int32_t *d_cnt, float *d_rref, void *d_ws,
                                md_stream_t stream);
/* Build every replica's neighbor rows from d_r [N][4]. */
JMD_API md_status md_batch_build(md_batch *bt, const float *d_r, uint32_t *d_status, md_stream_t stream);
/* Forces (w = per-particle energy) of every replica into d_f. */
JMD_API md_status md_batch_forces(md_batch *bt, const float *d_r, float *d_f, uint32_t *d_status, md_stream_t stream);
/* nsteps of velocity-Verlet NVE for every replica with its own dt, mass and
 * rebuild decisions (a replica rebuilds only when one of its particles
 * moved more than skin/2).  d_PE / d_KE (R x nsteps doubles, may be NULL):
 * per-replica FP64 energies after each step; v.w receives each particle's
 * kinetic energy.  Arithmetic per particle equals the single-system path
 * with md_set_pair_tpp(tpp), so each replica matches its own md_integrate_nve
 * run bit for bit.  use_graph: one graph launch with device loop control. */
JMD_API md_status md_batch_run_nve(md_batch *bt, float *d_r, float *d_v, float *d_f, int nsteps, double *d_PE,
                                   double *d_KE, int use_graph, uint32_t *d_status, md_stream_t stream);
/* Builds per replica since bind (synchronous). */
JMD_API md_status md_batch_stats(const md_batch *bt, uint32_t *h_builds, md_stream_t stream);
/* Pick the fastest threads-per-particle (4, 8, 16) by timing `probe` graph
 * steps of each on the caller's state (restored afterwards; d_scratch holds
 * 2 N float4); cached as JSON in cache_path (may be NULL) keyed by the
 * replica sizes and kinds.  Synchronous. */
JMD_API md_status md_batch_autotune(md_batch *bt, float *d_r, float *d_v, float *d_f, void *d_scratch, int probe,
                                    const char *cache_path, int *tpp_out, md_stream_t stream);

/* Threads per particle of the force kernel per replica: tpp_of_rep [R],
 * each 4, 8 or 16 (host array).  The force step then runs one launch per
 * distinct value over the particles of those replicas, listed in the
 * workspace (synchronous upload on `stream`).  NULL returns to one launch
 * with bt->tpp for all.  Each replica's arithmetic is that of the single-
 * system path with its own threads per particle.  Needs a bound batch;
 * MD_ERR_INVALID for other values. */
JMD_API md_status md_batch_set_class_tpp(md_batch *bt, const int *tpp_of_rep, md_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Status and accounting                                                     */
/* ------------------------------------------------------------------------ */
/* Synchronous: copies *d_status to *h_status after `stream` drains. */
JMD_API md_status md_status_poll(const uint32_t *d_status, uint32_t *h_status, md_stream_t stream);

/* Number of this library's kernels that have run in this process (graph
 * launches count every kernel node they ran).  Synchronizes the device. */
JMD_API uint64_t md_launch_count(void);

/* A single-thread device wait on *d_flag (nonzero ends it) bounded by
 * `limit` polls (at most 2^24, about 100 ns apart): on running out it ORs
 * MD_ERR_TIMEOUT into *d_status and returns, leaving the context usable.
 * The same bounded-wait rule guards every device wait in the library. */
JMD_API md_status md_bounded_wait(const uint32_t *d_flag, uint64_t limit, uint32_t *d_status, md_stream_t stream);

/* FP32 FMA throughput probe (measurement only, not a step of the path):
 * launches `blocks` x `threads` threads, each running 8 independent chains of
 * `iters` fused multiply-adds, and writes one float per thread to d_out
 * (caller-owned, blocks*threads floats).  *flops (host, may be NULL)
 * receives the FLOP count of the launch (an FMA counts 2).  Timing it with
 * events on `stream` gives the FP32 peak that ALU-bound kernels are compared
 * against.  MD_ERR_INVALID for a null d_out, blocks <= 0, iters <= 0 or
 * threads not a multiple of 32 in [32, 1024]. */
JMD_API md_status md_fma_probe(float *d_out, int blocks, int threads, int iters, uint64_t *flops, md_stream_t stream);

/* Library version string. */
JMD_API const char *md_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JMD_H */
