// fwi_internal.cuh -- plan layout and kernel argument blocks shared by the
// translation units of libfwi (host + device).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fwi.h"

namespace fwi {

constexpr int kStatusBytes = 256;   // status word region at the start of the workspace
// Threads per propagator CTA: the adjoint keeps two register arrays per
// thread (imaging accumulator and snapshot prefetch), so it runs with fewer,
// longer strips and up to 85 registers per thread.
constexpr int kMaxThreadsFwd = 1024;
constexpr int kMaxThreadsAdj = 768;
// Rows per thread strip of the fast (compile-time pitch) propagators.
constexpr int kFastRows = 22;
// Shared-memory pitch of the column-pair forward (even for 8-byte accesses;
// 11 x 162 = 22 (mod 32) keeps strip-straddling half-warps conflict-free).
constexpr int kPairPitch = 162;
constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// ---------------------------------------------------------------------------
// Propagator (forward / adjoint) launch shape for the SMEM-resident kernel:
// one CTA per (model, shot), each thread owns a column strip of `rows`
// consecutive padded rows at one padded column.
struct ResidentShape {
    int threads;     // blockDim.x (multiple of 32)
    int nstrip;      // strips per column
    int rows;        // rows per strip
    int maxrows;     // template bucket >= rows
    int chunk;       // time steps per staging chunk
    size_t smem;     // dynamic shared memory bytes
};

// Cluster propagators: a (model, shot) grid split by rows over up to
// kClusterCTAs CTAs of one cluster; shared-memory row pitch (compile time;
// padded widths up to kCluPitch - 4)
constexpr int kClusterCTAs = 8;
constexpr int kCluPitch = 341;
// threads per CTA of the cluster kernels with RS rows a thread (one CTA per
// SM): 21 warps put 6 on some scheduler, whose 16K registers then give 80 a
// thread, as 24 warps do
__host__ __device__ constexpr int clu_max_threads(int RS) { return RS > 13 ? 672 : 768; }
// column-pair cluster kernels: shared-memory row pitch (even: 8-byte rows),
// rows a thread, threads at most; the record keeps the pitch kCluPitch - 1
constexpr int kCluPairPitch = 342;
constexpr int kCluPairRows = 10;
constexpr int kCluPairThreads = 672;

struct ClusterArgs {
    int P;          // shared-memory row pitch
    int C;          // CTAs per cluster (2..kClusterCTAs)
    int RC;         // grid rows per CTA = nstrip * RS
    int RS;         // rows per thread strip
    int nstrip;     // strips per column
    int NXp;        // row pitch of the imaging sums in global memory
    int chunk;      // staged time steps
    float *acc;     // adjoint: imaging sums [bs][NZ][NXp] (to the fold)
    float *acc_src; // adjoint: source-cell sums [bs]
    int withhold;   // 1: send no halo rows (the bounded-wait self-check)
    unsigned long long wait_ns;   // bound of one halo wait
    int pair;       // 1: column-pair kernels (RS = kCluPairRows rows of two columns a thread)
};

struct Plan {
    fwi_problem p;           // copy; index pointers below replace the caller's
    fwi_w2_params w2;
    int NZ, NX;
    double t0;
    int src_pz[FWI_MAX_SHOTS], src_px[FWI_MAX_SHOTS];   // padded coordinates
    int rec_pz[FWI_MAX_RECEIVERS], rec_px[FWI_MAX_RECEIVERS];
    ResidentShape shape;       // forward propagator
    ResidentShape shape_adj;   // adjoint propagator
    bool fast;                 // compile-time pitch kernels (else the generic ones)
    bool tiled;                // global-memory tiled kernels (grids beyond shared memory)
    bool cluster;              // cluster kernels for the store-all passes of a tiled plan
    bool cpml;                 // convolutional PML absorber (its own global-memory kernels)
    size_t ws_c;               // CPML: workspace offset of its fields and tables
    ClusterArgs clu;           // their shape
    int clu_threads, clu_chunk_fwd, clu_chunk_adj;
    int NXp;                   // tiled: row pitch of the fields (NX rounded up to 4)
    int rec_pitch;             // row pitch of a record plane
    bool fwd_pair;             // forward on column pairs (even padded width)
    bool adj_pair;             // adjoint on column pairs (same condition)
    int tile_rows;             // tiled, scalar threads: rows a thread (8 or 4)
    bool tile_quads;           // tiled: four columns x 2 rows a thread, 16-byte accesses (default)
    int fast_P, fast_PR, fast_NZM;  // their shared-memory pitch, record pitch, row capacity
    int nzs;                   // rows of one wavefield-record plane (>= NZ)
    // byte offsets inside the caller buffers
    size_t ws_w2, ws_gshot, ws_bytes;
    size_t ctx_M, ctx_S, ctx_S2, ctx_cshift, ctx_str, ctx_omega, ctx_Qb, ctx_Qf, ctx_bytes;
    size_t snap_bytes;
    // checkpoint + recompute: every ckpt_every steps (0: store-all record)
    int ckpt_every, nslot;
    size_t ws_seg, ws_astate, ws_asrc;    // workspace: segment record, adjoint state
    // tiled path: fields, adjoint levels and sums, per-model tables
    size_t ws_t_u0, ws_t_u1, ws_t_v, ws_t_p0, ws_t_p1, ws_t_w, ws_t_acc, ws_t_ka, ws_t_ab,
        ws_t_accsrc, ws_t_rec, ws_t_src;
};

// ---------------------------------------------------------------------------
// Argument block of the propagator kernels (passed as a __grid_constant__
// parameter; geometry tables travel inside it, so no device allocation is
// needed for them).
struct PropArgs {
    int nz, nx, nb, NZ, NX, nt, ns, nr;
    int nzs;                             // rows of one wavefield-record plane
    int units;                           // (model, shot) units of the plan: batch x ns
    int rows, nstrip, chunk;
    float dt;
    double dtd, t0d;                     // dt and the Ricker delay in double: the
                                         // per-cell coefficients and the source
                                         // times are formed in double, rounded once
    double ex0d, ez0d;                   // eta0 * dt / 2 per axis, double
    float c0, cx1, cx2, cz1, cz2;        // Laplacian weights divided by h^2
    float2 w2[5];                        // the same weights in pairs (c0, cx1, cx2, cz1,
                                         // cz2), operands of the packed instructions
    float ex0, ez0;                      // eta0 * dt / 2 per axis
    float inv_nb;
    float fp, t0, src_scale;             // Ricker and 1/(dx dz)
    float vmax;
    const float *v;                      // [B][nz][nx]
    float *d_syn;                        // forward: [B][ns][nr][nt]
    float *snap;                         // forward: written (may be null); adjoint: read
    const float *adj;                    // adjoint: [B][ns][nr][nt]
    float *gshot;                        // adjoint: [B][ns][nz][nx]
    int *status;
    // Time window of this launch (checkpointed runs split the time loop):
    // forward steps [j_begin, j_end), or adjoint steps [j_begin, j_end).
    int j_begin, j_end;
    // Record plane of forward step f is f - rec_base inside a block of
    // rec_planes planes per (model, shot).
    int rec_base, rec_planes;
    // Forward: state to resume from at j_begin ([B*ns][2][NZ][NX]; null =
    // start from rest), and checkpoint slots written at every multiple of
    // ckpt_every ([nslot][B*ns][2][NZ][NX]; null = none).
    const float *resume;
    float *ckpt;
    int ckpt_every;
    // Adjoint: state carried between windows ([B*ns][3][NZ][NX]: level j,
    // level j-1, imaging sums) and the source-cell imaging sum ([B*ns]).
    float *astate, *asrc;
    int16_t src_pz[FWI_MAX_SHOTS], src_px[FWI_MAX_SHOTS];
    int16_t rec_pz[FWI_MAX_RECEIVERS], rec_px[FWI_MAX_RECEIVERS];
};

// Persistent launch over the (model, shot) units of several resident
// column-pair plans (k_fwd_pair_queue / k_adj_pair_queue): plan p owns units
// start[p] .. start[p+1]-1, CTAs draw unit numbers from *counter
constexpr int kQueuePlans = FWI_QUEUE_MAX_PLANS;
struct QueueArgs {
    int n, total;
    int start[kQueuePlans + 1];
    int *counter;
    PropArgs a[kQueuePlans];
};

PropArgs make_args(const Plan &pl);
__global__ void k_shot_sum(int B, int ns, int n, const float *__restrict__ gshot,
                           float *__restrict__ grad);
// Whether a plan can take part in a persistent launch (store-all resident
// column-pair plans of the 110-row bucket)
bool queue_ok(const Plan &pl);
// Whether two plans share spacing, time step, layer, top boundary and source
// (a persistent launch takes its time-loop coefficients from its first plan)
bool queue_same_physics(const Plan &a, const Plan &b);
// One persistent launch of the forward (adj false; a[i] with v, d_syn, snap,
// status set) or adjoint (adj true; v, adj, snap, gshot, status set) of the
// plans, on at most one CTA per SM; *counter is zeroed first
cudaError_t launch_fast_queue(const Plan *const *plans, int n, bool adj, const PropArgs *a,
                              int *counter, cudaStream_t st);

// Records the message returned by fwi_last_error() for the calling thread
// and returns code.
fwi_status record_error(fwi_status code, const char *fmt, ...);

// Status codes the device writes (first error wins).
__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

// One launch's share of a checkpointed run (defaults: the whole time loop,
// records indexed by absolute step, no state carried).
struct Window {
    int j_begin = 0, j_end = -1;          // -1: nt
    int rec_base = 0, rec_planes = -1;    // -1: nt
    const float *resume = nullptr;
    float *ckpt = nullptr;
    int ckpt_every = 0;
    float *astate = nullptr, *asrc = nullptr;
    bool wait_check = false;              // cluster / tiled kernels: withhold the halos
};

// Launchers (return cudaGetLastError() of the launches they made).
// `workspace` is the caller's workspace (status word at its start).
cudaError_t launch_forward(const Plan &pl, const float *v, float *d_syn, float *snap,
                           void *workspace, cudaStream_t st, const Window &w = Window());
// Adjoint over one window; the gradient is folded and written to gshot when
// the window ends at nt (and then summed over shots into grad if grad is set).
cudaError_t launch_adjoint(const Plan &pl, const float *v, const float *adj,
                           const float *snap, float *grad, float *gshot, void *workspace,
                           cudaStream_t st, const Window &w = Window());
cudaError_t launch_w2_prepare(const Plan &pl, const float *d_obs, unsigned char *ctx,
                              cudaStream_t st);
cudaError_t launch_w2_misfit(const Plan &pl, const unsigned char *ctx, const float *d_syn,
                             float *J, float *w2_out, float *adj, float *w2_scratch,
                             cudaStream_t st);
cudaError_t launch_guided(int B, int nz, int nx, const fwi_guide_params &gp,
                          const float *vprime, const float *v0hat, const float *g,
                          const float *h, float *vout, float *rho, cudaStream_t st);

// Host-side choice of the resident launch shape; returns false if the grid
// does not fit the shared-memory resident kernel.
bool choose_resident_shape(int NZ, int NX, int nr, bool adj, ResidentShape *out);

// Fast propagators: bucket (pitch, row capacity) for a padded grid, their
// shared memory, and their launch.
bool fast_bucket(int NZ, int NX, int *P, int *PR, int *NZM);
size_t fast_smem(int P, int NZM, bool adj, int chunk, int nr);
int fast_chunk(int P, int NZM, bool adj, int nr);   // staging steps that fit (<= 32; 0: none)
bool fwd_pair_ok(int NX, int NZ, int NZM);
cudaError_t launch_fast(const Plan &pl, bool adj, const PropArgs &a, cudaStream_t st);
// Cluster propagators (whole time loop, store-all plans): shared memory of
// one CTA, and the launch
size_t cluster_smem(int RC, int P, bool adj, int chunk, int nr, bool pair = false);
cudaError_t launch_cluster(const Plan &pl, bool adj, const PropArgs &a, unsigned char *ws,
                           cudaStream_t st, bool wait_check = false);
cudaError_t launch_tile_fold(const Plan &pl, const PropArgs &a, unsigned char *ws,
                             cudaStream_t st);
// CPML propagators (absorber = FWI_ABSORBER_CPML): workspace bytes of their
// fields and tables, and the whole forward or adjoint time loop
size_t cpml_workspace(const Plan &pl);
cudaError_t launch_cpml(const Plan &pl, bool adj, const PropArgs &a, unsigned char *ws,
                        cudaStream_t st);
// Tiled propagators: one launch per step over [a.j_begin, a.j_end)
cudaError_t launch_tiled(const Plan &pl, bool adj, const PropArgs &a, unsigned char *ws,
                         cudaStream_t st, bool wait_check = false);

}  // namespace fwi
