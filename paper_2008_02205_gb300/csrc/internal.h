// Internal declarations of the MLPG transport library (host + device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "mlpg.h"

#define MLPG_MAX_DIR 1024   // directions per problem (one thread per direction in a block row)
#define MLPG_MAX_RESTART 32 // restart length cap (Gram-Schmidt keeps one accumulator per basis vector in registers)
#define MLPG_MAX_CELL_FUNCS 40  // functions whose support can reach one 2D cell
#define MLPG_BLOCK_PTS 16       // points per block of the block-Jacobi preconditioner

namespace mlpg {

// error helpers --------------------------------------------------------------
#define MLPG_TRY(expr)                         \
    do {                                       \
        mlpg_status _s = (expr);               \
        if (_s != MLPG_OK) return _s;          \
    } while (0)

mlpg_status cuda_fail(mlpg_ctx *ctx, cudaError_t e, const char *what, const char *file, int line);
#define CU(ctx, expr)                                                               \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) return mlpg::cuda_fail((ctx), _e, #expr, __FILE__, __LINE__); \
    } while (0)
#define CU_LAUNCH(ctx)               \
    do {                             \
        (ctx)->st.kernel_launches++; \
        CU(ctx, cudaGetLastError()); \
    } while (0)

// host geometry (geometry.cpp) ----------------------------------------------
constexpr int32_t kLabelExtent = -100;
// 3D cells as flat element lists: tetrahedra (generator of `owner`, three
// stored vertices) and boundary triangles (three stored vertices, box face).
struct HostCells3 {
    std::vector<double> volume;      // n
    std::vector<int32_t> tet_owner;  // ntet
    std::vector<double> tet_v;       // 9 * ntet
    std::vector<int32_t> tri_owner;  // ntri
    std::vector<int32_t> tri_face;   // ntri: 0..5 = -x, +x, -y, +y, -z, +z
    std::vector<double> tri_v;       // 9 * ntri
};
int64_t build_cells_3d(int64_t n, const double *x, const double *R, const double *lo,
                       const double *hi, const int32_t *rowptr, const int32_t *col, HostCells3 &out);
// Row tiles of the batched L-apply (tiles.cpp): Morton-consecutive rows, the
// halo (union of their columns) and sliced-ELL record slots.
struct TileLayout {
    int rows_per_tile = 0;
    int64_t ntile = 0;
    std::vector<int64_t> base;    // ntile + 1: first record slot of each tile
    std::vector<int32_t> width;   // ntile: entries per row slot (longest row of the tile, rounded up)
    std::vector<int32_t> row;     // ntile * rows_per_tile: row of each row slot, -1 past n
    std::vector<int64_t> hptr;    // ntile + 1: halo ranges in hcol
    std::vector<int32_t> hcol;    // halo columns, sorted within each tile
    std::vector<int32_t> perm;    // record slot -> pattern entry, -1 for padding
    std::vector<int32_t> lcol;    // record slot -> halo index of its column (0 for padding)
    int64_t max_halo = 0;
    int32_t max_width = 0;
};
// order[n]: the rows in tile order.  Returns the number of record slots.
int64_t build_tiles(int64_t n, const int32_t *rowptr, const int32_t *col, const int32_t *order, int rows_per_tile,
                    int width_multiple, TileLayout &out);
// Reference rules (quadrature.cpp).
void gauss_jacobi_newton(int n, double a, double b, double *t, double *w);
void triangle_rule(int n1d, double *xi /*2*n1d^2*/, double *w);
void tet_rule(int n1d, double *xi /*3*n1d^3*/, double *w);
void line_rule(int n, double *t, double *w);

// GMRES workspace ------------------------------------------------------------
template <typename T>
struct Gmres {
    int64_t n = 0;
    int M = 0, R = 0;
    T *V = nullptr;        // (R + 1) * n * M
    T *Z = nullptr;        // n * M: preconditioned basis vector
    T *W = nullptr;        // n * M: scratch for true residuals
    double *H = nullptr;   // M * (R + 1) * R
    double *cs = nullptr, *sn = nullptr;   // M * R
    double *g = nullptr;   // M * (R + 1)
    double *h = nullptr;   // (R + 1) * M : dot results of the current step
    double *h2 = nullptr;  // (R + 1) * M
    double *y = nullptr;   // R * M
    float *y32 = nullptr;  // R * M: float copy of y
    double *bnorm = nullptr, *beta = nullptr, *resid = nullptr;  // M
    double *nrm2 = nullptr;  // M: squared norms of the current vector
    int *active = nullptr; // M: 1 while iterating in this cycle
    int *kcol = nullptr;   // M: Arnoldi columns used in this cycle
    int *its = nullptr;    // M: total iterations
    double *partial = nullptr; // reduction partials
    int64_t partial_cap = 0;
    int *h_active = nullptr;   // pinned host mirror: number of active directions
    int *d_active_count = nullptr;
    bool reorth = true;        // CGS2 (true) or a single classical Gram-Schmidt pass
    int its_slot = 0;          // iteration counter of the step this solve adds to (0 inner, 1 outer, 2 diffusion)
    T *Zf = nullptr;           // R * n * M: preconditioned basis vectors (flexible GMRES), or null
};

}  // namespace mlpg

struct mlpg_ctx {
    mlpg_options opt{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int state = 0;  // 0 created, 1 integrated, 2 assembled
    int64_t n = 0;
    int m = 0, dim = 2;
    std::vector<void *> allocs;       // device allocations
    std::vector<void *> host_allocs;  // pinned host allocations

    // inputs (device)
    double *x = nullptr, *R = nullptr, *V = nullptr, *sig_t = nullptr, *sig_s = nullptr,
           *q = nullptr, *omega = nullptr, *w = nullptr, *tau = nullptr;
    std::vector<double> h_x, h_R, h_omega, h_w;
    double psi_b[6] = {0, 0, 0, 0, 0, 0};
    bool have_initial = false;

    // connectivity
    int64_t nnz = 0;
    int32_t *rowptr = nullptr, *col = nullptr, *diag = nullptr;
    std::vector<int32_t> h_rowptr, h_col;

    // cells
    int64_t nverts = 0, nvq = 0, nbq = 0;
    int32_t *cptr = nullptr, *labels = nullptr;
    double *verts = nullptr;
    // 3D cells as elements: tetrahedra and boundary triangles (HostCells3)
    int64_t ntet = 0, nbtri = 0;
    int32_t *tet_owner = nullptr, *tri_owner = nullptr, *tri_face = nullptr;
    double *tet_v = nullptr, *tri_v = nullptr;
    double *interp = nullptr;   // [nnz]: V_j U_j(x_i) on the overlap pattern
    int *d_flag = nullptr;      // device error flag (assembly / RK)

    // integrated forms (FP64)
    double *mats = nullptr, *vecs = nullptr;
    int nmats = 0, nvecs = 0;

    // operators for the current 1/(c dt)
    double kappa = -1.0;
    double *A64 = nullptr;      // [6][nnz] direction-independent LHS arrays
    double *L64 = nullptr;      // [nnz][m] materialised per-direction L_m (FP64 path)
    float *A32 = nullptr;       // [6][nnz]
    int64_t nb = 0;             // boundary-segment entries
    int32_t *bptr = nullptr, *bcol = nullptr;
    int32_t *brow = nullptr;    // rows with face terms (nbrow of them)
    int64_t nbrow = 0;
    float *bval32 = nullptr;    // [2 dim][nb]
    double *bval64 = nullptr;   // [2 dim][nb]
    double *coef = nullptr;     // [m][8]: 1, Ox, Oy, Ox^2, Oy^2, OxOy, (unused x2)
    double *fcoef = nullptr;    // [m][2 dim]: max(Omega . n_f, 0)
    float *coef32 = nullptr;    // [m][16]: float copy of coef (0..7) and fcoef (8..11)
    double *dinv64 = nullptr;   // [n][m]
    float *dinv32 = nullptr;
    double *r64 = nullptr;      // [n][m] boundary + volume source
    double *T64 = nullptr;      // [3][nnz]: kappa M0, kappa tau G^x, kappa tau G^y
    double *S64 = nullptr;      // [3][nnz]: Ms, tau Gs^x, tau Gs^y

    // state and work
    double *Psi = nullptr, *Phi = nullptr;   // [n][m], [n]
    double *f64 = nullptr, *res64 = nullptr, *tmp64 = nullptr;  // [n][m]
    double *bpsi64 = nullptr;                // [n][m]
    float *rhs32 = nullptr, *sol32 = nullptr, *bpsi32 = nullptr;  // [n][m]
    double *rhs64b = nullptr, *sol64 = nullptr;   // [n][m]
    double *nvec = nullptr;                  // [8][n] small n-vectors
    double *red = nullptr;                   // reduction scratch
    int64_t red_cap = 0;
    double *h_red = nullptr;                 // pinned host scalars

    mlpg::Gmres<double> g64;
    mlpg::Gmres<float> g32;
    mlpg::Gmres<double> gout;
    mlpg::Gmres<double> gdsa;     // diffusion solves of the DSA-like outer preconditioner

    // DSA-like outer preconditioner: diffusion operator on the pattern and its block inverses
    double *Cdiff = nullptr;      // [nnz] FP64
    double *Cinv = nullptr;       // [nblk][kBlockPts][kBlockPts] FP64
    double *dsa_buf = nullptr;    // [2][n] work vectors

    double ops_psib[6] = {0, 0, 0, 0, 0, 0};  // inflow the operators were formed with
    int32_t *rowidx = nullptr;  // [nnz] row of each pattern entry
    double *abc = nullptr;      // [3][n] MS partial products

    // block-Jacobi preconditioner: Morton-ordered blocks of kBlockPts points
    int64_t nblk = 0;
    int32_t *bmember = nullptr; // [nblk * kBlockPts] point of each block slot (-1: empty)
    int32_t *bof = nullptr;     // [n] block * kBlockPts + slot of each point
    std::vector<int32_t> h_order;  // [n] points in Morton order (host)

    // row tiles of the FP32 L-apply (tiles.cpp), used when m % 4 == 0
    int tile_rows = 0, tile_chunk = 0, tile_dpt = 0, tile_xs = 0;  // rows per tile, directions per CTA, per thread, smem row stride
    bool tile_mma = false;      // the tensor-core variant of the tiled apply (apply_kernel 3)
    bool tile_gather = false;   // tiles with X read from global memory, no staged halo (apply_kernel 4)
    int64_t ntile = 0, nslot = 0;
    size_t tile_smem = 0;       // dynamic shared memory of the tiled kernel: halo rows + record stages
    int tile_xs_f4 = 0;         // float4 words of the staged halo (the record stages follow)
    int64_t tile_max_halo = 0;  // largest halo of a tile
    int *d_tile_err = nullptr;  // set by a tile-kernel wait that gave up (bounded waits)
    int32_t *t_base = nullptr, *t_width = nullptr, *t_row = nullptr, *t_hptr = nullptr, *t_hcol = nullptr;
    int32_t *t_perm = nullptr, *t_lcol = nullptr;
    int32_t *t_bhalo = nullptr;  // [nb]: halo offset (index x tile_xs) of each boundary-segment entry's column
    float *t_rec = nullptr;     // [nslot][rec words]: the base-array values of each slot, then its halo index
    float *Pinv = nullptr;      // [nblk][kBlockPts][kBlockPts][m] inverse diagonal blocks of L_m
    uint16_t *Pinv16 = nullptr; // same, FP16 bits scaled by Pscale^-1 (mixed mode), or null
    float *Pscale = nullptr;    // [nblk][m] power-of-two decode factor of each FP16 block
    double cur_inner_tol = 0.0; // tolerance of the inner solves inside the outer operator
    long long *d_its = nullptr;  // [3] inner / outer / diffusion Krylov iterations of the current step (device)
    void *bank64 = nullptr, *bank32 = nullptr;  // inner solutions of the outer basis (+ accumulator)
    double *hist[2] = {nullptr, nullptr};       // previous states for the initial guess
    int nhist = 0;                              // how many of them are valid

    // direction shards: cross-shard sum callback and its pinned host buffer
    mlpg_reduce_fn reduce_fn = nullptr;
    void *reduce_user = nullptr;
    double *reduce_host = nullptr;   // n + 8 doubles

    // stats
    mlpg_stats st{};
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    int ev_used = 0;
};

namespace mlpg {
mlpg_status set_err(mlpg_ctx *ctx, mlpg_status s, const std::string &msg);
template <typename T>
mlpg_status dalloc(mlpg_ctx *ctx, T **p, size_t count) {
    void *q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, MLPG_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    ctx->allocs.push_back(q);
    ctx->st.device_bytes += (int64_t)(count * sizeof(T));
    *p = static_cast<T *>(q);
    return MLPG_OK;
}

// kernels / launchers (neighbors.cu, assemble.cu, operators.cu, krylov.cu)
mlpg_status run_neighbors(mlpg_ctx *ctx);
mlpg_status run_cells_2d(mlpg_ctx *ctx, int tri_points, int line_points);
mlpg_status run_cells_3d(mlpg_ctx *ctx);   // cells3d.cu: element lists and volumes on the device
mlpg_status run_interp(mlpg_ctx *ctx);
mlpg_status run_assemble(mlpg_ctx *ctx);
mlpg_status run_interp_3d(mlpg_ctx *ctx);
mlpg_status run_assemble_3d(mlpg_ctx *ctx);
mlpg_status form_operators(mlpg_ctx *ctx, double kappa);
mlpg_status apply_L64(mlpg_ctx *ctx, const double *X, double *Y);
mlpg_status apply_L32(mlpg_ctx *ctx, const float *X, float *Y);
mlpg_status step_fp64(mlpg_ctx *ctx, double dt);
mlpg_status step_mixed(mlpg_ctx *ctx, double dt);
mlpg_status apply_L64_res(mlpg_ctx *ctx, const double *X, const double *B, double *Y);
mlpg_status apply_L32_res(mlpg_ctx *ctx, const float *X, const float *B, float *Y);
mlpg_status rhs_T(mlpg_ctx *ctx, const double *Psi_prev, double *F);
template <typename T>
mlpg_status apply_MS(mlpg_ctx *ctx, const double *phi, T *out);
mlpg_status interp_flux(mlpg_ctx *ctx, double *out_dev, int kind);
// z = P^{-1} v (block-Jacobi); with sc != null, v is first scaled in place by sc[direction]
template <typename T>
mlpg_status apply_prec(mlpg_ctx *ctx, T *v, T *z, const double *sc);
mlpg_status build_blocks(mlpg_ctx *ctx);
// Direction shards (api.cu): replace count partial sums by the sums over all
// shards (a no-op without a callback).  shard_sum_dev works on a device vector
// (synchronises the stream), shard_sum_host on host values.
mlpg_status shard_sum_dev(mlpg_ctx *ctx, double *dev, int64_t count);
mlpg_status shard_sum_host(mlpg_ctx *ctx, double *host, int64_t count);
// DSA-like outer preconditioner (operators.cu): C for 1/(c dt) = kappa, y = C x or B - C x,
// y = Ms x, and z = blockJacobi(C)^{-1} v (v first scaled in place by sc[0] when sc != null)
mlpg_status form_diffusion(mlpg_ctx *ctx, double kappa);
mlpg_status apply_C(mlpg_ctx *ctx, const double *X, const double *B, double *Y);
mlpg_status apply_Ms_scalar(mlpg_ctx *ctx, const double *X, double *Y);
mlpg_status apply_Cprec(mlpg_ctx *ctx, double *v, double *z, const double *sc);
void harvest_timing(mlpg_ctx *ctx);
}  // namespace mlpg
