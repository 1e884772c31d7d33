// Internal declarations shared by the CUDA kernels and the host orchestration.
// Nothing here is part of the C ABI (include/sg.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace sg {

// Geometry and boundary description of one multigrid level.  Arrays are dense
// [nz][ny][nx] (x fastest) without ghost cells; the ghost values of Sec. 2.3 are
// produced on the fly by the kernels:
//   periodic axis           -> the cell on the opposite side (Eq. periodic)
//   Dirichlet with faces    -> 2 * face - active              (Eq. solution_ghost)
//   Dirichlet without faces -> -active                        (Eq. error_ghost)
struct LevelGeom {
    int nx, ny, nz;
    double ihx2, ihy2, ihz2;          // 1 / h_d^2
    float ihx2f, ihy2f, ihz2f;        // the same in FP32: FP32 kernels must never convert from FP64
                                      // (GB300 issues FP64 and its conversions at 1/64 of the FP32 rate)
    int per[3];                       // periodic flag per axis (x, y, z)
    const double* face[6];            // -x,+x,-y,+y,-z,+z or all nullptr (homogeneous)
    int twod;                         // a two-dimensional level (Sec. 2.2): nz = 1, z periodic, 1 / h_z^2 = 0,
                                      // so the seven-point kernels compute the five-point operator exactly;
                                      // restriction averages 4 cells, prolongation weighs 9/3/3/1
};

// 1 / h^2 per axis in the kernel's precision.
template <typename T> __host__ __device__ __forceinline__ T ih2x(const LevelGeom& g);
template <> __host__ __device__ __forceinline__ float ih2x<float>(const LevelGeom& g) { return g.ihx2f; }
template <> __host__ __device__ __forceinline__ double ih2x<double>(const LevelGeom& g) { return g.ihx2; }
template <typename T> __host__ __device__ __forceinline__ T ih2y(const LevelGeom& g);
template <> __host__ __device__ __forceinline__ float ih2y<float>(const LevelGeom& g) { return g.ihy2f; }
template <> __host__ __device__ __forceinline__ double ih2y<double>(const LevelGeom& g) { return g.ihy2; }
template <typename T> __host__ __device__ __forceinline__ T ih2z(const LevelGeom& g);
template <> __host__ __device__ __forceinline__ float ih2z<float>(const LevelGeom& g) { return g.ihz2f; }
template <> __host__ __device__ __forceinline__ double ih2z<double>(const LevelGeom& g) { return g.ihz2; }

// Per-stage coefficients of one RKL stage (App. A, Eq. RKL_intermediate_source).
//   first stage : z = tau (L Y0 - f);  Y1 = Y0 + mut1 * z;   (RKL2 stores z as Z0)
//   later stages: Yj = mu Y_{j-1} + nu Y_{j-2} + mut_tau (L Y_{j-1} - f)
//                      [RKL2: + c0 Y0 + gt Z0]
struct StageCoef {
    double tau;       // first stage only
    double mut1;      // first stage only: mu~_1
    double mu, nu;
    double mut_tau;   // mu~_j * tau
    double c0;        // 1 - mu_j - nu_j (RKL2)
    double gt;        // gamma~_j (RKL2; multiplies Z0 = tau (M Y0 - f))
};

// Deterministic two-pass reductions: kernels write one Partial per block, a
// single-block kernel folds them in a fixed order into a Reduced.
struct Partial {
    double sumsq;     // sum of r^2
    double maxabs;    // max |r|
    double sum;       // sum of a secondary field (coarse rhs for the periodic mean)
    double pad;
};
struct Reduced {
    double sumsq, maxabs, sum, count;
};

constexpr int kRedThreads = 256;

// ---- launchers (kernels_stencil.cu) ----------------------------------------
// Number of blocks (= Partial slots) a residual / residual-restrict launch uses.
long long residual_blocks(const LevelGeom& g);
long long residual_zero_blocks(const LevelGeom& g);   // launch_residual_zero, both passes
long long restrict_blocks(const LevelGeom& g);
constexpr long long kSumBlocks = 152LL * 8;     // grid of the 1D reduction kernels

template <typename T>
cudaError_t launch_stage(const LevelGeom& g, int order, bool first, const StageCoef& c,
                         const T* ym1, const T* ym2, const T* y0, const T* z0, const T* rhs,
                         T* out, T* z0_out, cudaStream_t st);

// One colour (0: (i + j + k) even, 1: odd) of a red-black Gauss-Seidel / SOR
// sweep of L u = rhs, in place (periodic extents must be even).
template <typename T>
cudaError_t launch_gsrb(const LevelGeom& g, int colour, double omega, T* u, const T* rhs, cudaStream_t st);

// r = rhs - L u (TI), optionally stored as TO (r_out) and in full precision
// (r_full), block partials of sum r^2 / max|r|.
template <typename TI, typename TO>
cudaError_t launch_residual(const LevelGeom& g, const TI* u, const TI* rhs, TO* r_out,
                            Partial* partials, int* nblocks_out, cudaStream_t st, TI* r_full = nullptr);
// The same for u = 0 (FP64 rhs): r = rhs - L 0, the face terms only
// (*nkernels: the kernels it launched, one or two).
template <typename TO>
cudaError_t launch_residual_zero(const LevelGeom& g, const double* rhs, TO* r_out, Partial* partials,
                                 int* nblocks_out, cudaStream_t st, double* r_full = nullptr,
                                 int* nkernels = nullptr);

// Fused residual + 8-cell restriction (+ norm partials, + coarse sum partials).
template <typename T>
cudaError_t launch_residual_restrict(const LevelGeom& fine, const T* u, const T* rhs,
                                     T* coarse_out, Partial* partials, int* nblocks_out,
                                     cudaStream_t st);

// fine += P(coarse) with coarse ghosts by the homogeneous/periodic rule.
template <typename T>
cudaError_t launch_prolong_correct(const LevelGeom& fine, const T* coarse, T* fine_u,
                                   cudaStream_t st);

cudaError_t launch_finalize(const Partial* partials, int n, Reduced* out, cudaStream_t st);

// The FP64 residual r = rhs - A u (r into r_full, its FP32 copy into r_out,
// the norms of the copy into partials) with the neighbour sum in exact 64-bit
// fixed point: a pre-pass writes the scale into *scratch (one word on the
// device), then the residual (*nkernels: the kernels launched, two; one, the
// FP64 residual, for levels that are not strips of four cells).
cudaError_t launch_residual_exact(const LevelGeom& g, const double* u, const double* rhs, float* r_out,
                                  double* r_full, Partial* partials, unsigned* scratch, int* nblocks_out,
                                  int* nkernels, cudaStream_t st);
// phi += e (FP64) and r64 -= A_0 e (FP64 residual by recurrence, A_0 e summed
// error-free in FP32), r32 = r64 rounded, block partials of |r32|.
cudaError_t launch_update_residual(const LevelGeom& g, double* phi, const float* e, double* r64, float* r32,
                                  Partial* partials, int* nblocks_out, cudaStream_t st);

template <typename T>
cudaError_t launch_subtract_mean(T* x, long long n, const Reduced* red, cudaStream_t st);

cudaError_t launch_scale_copy(const double* src, double* dst, double scale, long long n,
                              cudaStream_t st);
// dst = scale src (or a plain copy when !scaled) where src or dst is pinned
// host memory mapped into the device address space.
cudaError_t launch_link_copy(const double* src, double* dst, double scale, bool scaled, long long n,
                             cudaStream_t st);
cudaError_t launch_add_f32_to_f64(double* phi, const float* e, long long n, cudaStream_t st);
cudaError_t launch_sub_mean_f64(double* x, long long n, const Reduced* red, cudaStream_t st);
cudaError_t launch_sum_partials_f64(const double* x, long long n, Partial* partials,
                                    int* nblocks_out, cudaStream_t st);

// ---- FP64 throughput probe (kernels_probe.cu) -------------------------------
// TFLOP/s of FP64 FMA chains on every SM of the current device (2 flops per FMA).
cudaError_t probe_fp64_rate(double* tflops, double* ms);

// ---- the convergence loop on the device (kernels_loop.cu) -------------------
constexpr int kLoopHistory = 256;          // entries of the residual history kept (SG_MAX_HISTORY)
constexpr int kLoopRunning = 0, kLoopDone = 1, kLoopNotConverged = 2, kLoopNonFinite = 3;
// State of one solve's cycle loop in device memory: set by the host before
// the solve graph is launched, read back once when it has finished.
struct DeviceLoop {
    double rden;            // ||L 0 - f|| (1 if zero)
    double nn;              // cells of level 0
    double tol;             // relative L2 tolerance
    double mtol;            // > 0: stop on max |r| <= mtol instead
    int limit;              // cycle cap (or the fixed count)
    int fixed;              // run exactly `limit` cycles
    int confirm;            // mixed precision: confirm a met recurrence residual in FP64
    int m;                  // cycles run
    int status;             // kLoop*
    int pending;            // the inner loop ended for a confirmation
    int sched_len;          // entries of the coarse schedule
    int confirms;           // times the inner loop ended (the confirmation step ran)
    long long coarse_cells; // cells of the coarsest level
    long long coarse_stage_cells;   // sum over cycles of coarse cells x stages
    double rel, maxabs;     // the last recorded residual
    double history[kLoopHistory];
    int coarse_ss[kLoopHistory];
};
cudaError_t launch_loop_init(const DeviceLoop* d, cudaGraphConditionalHandle outer, cudaGraphConditionalHandle inner,
                             cudaStream_t st);
cudaError_t launch_loop_step(DeviceLoop* d, const Reduced* red, const int* ss_done, const int* sched,
                             cudaGraphConditionalHandle inner, cudaStream_t st);
cudaError_t launch_loop_confirm(DeviceLoop* d, const Reduced* red, cudaGraphConditionalHandle outer,
                                cudaGraphConditionalHandle inner, cudaStream_t st);

// ---- fused super-step, FP32 (kernels_fused.cu) -----------------------------
constexpr int kFusedMaxS = 6;
struct FusedCoef {
    float tau, mut1;                        // first stage
    float mu[kFusedMaxS + 1], nu[kFusedMaxS + 1], mut_tau[kFusedMaxS + 1];
    float c0[kFusedMaxS + 1], gt[kFusedMaxS + 1];
};
// True if the fused kernel handles (order, s): 2 <= s <= kFusedMaxS.
bool fused_supported(int order, int s);
cudaError_t fused_configure();
// out = Y_s of one super-step from y0 (nullptr: Y0 = 0) with homogeneous or
// periodic ghosts; out must not alias y0.
// tile_rows: 14 or 16 fixes the tile of the s = 2, 3 kernel; 0 lets its cost
// model choose.  tma: that kernel stages planes by tensor-map box copies where
// the level allows it (otherwise by per-strip copies).
cudaError_t launch_superstep_fused(const LevelGeom& g, int order, int s, bool zero_y0, const FusedCoef& cf,
                                   const float* y0, const float* f, float* out, cudaStream_t st,
                                   int tile_rows = 0, bool tma = false);
// s = 2, 3: stage-balanced variant with reflected halos (kernels_superstep.cu).
cudaError_t lean_configure();
cudaError_t launch_superstep_lean(const LevelGeom& g, int order, int s, bool zero_y0, const FusedCoef& cf,
                                  const float* y0, const float* f, float* out, cudaStream_t st, int tile_rows,
                                  bool tma);
// Launches of the TMA path that gave up a bounded wait (or found their shared
// memory misaligned) since the library was loaded; each wrote a NaN into its
// output, so the solve that ran it reports a non-finite residual.
unsigned lean_wait_failures();

// ---- coarsest-level solver (kernels_coarse.cu) -----------------------------
struct CoarseParams {
    LevelGeom g;          // homogeneous
    const void* rhs;      // level rhs (T)
    void* u_out;          // result (T)
    const int* sched;     // s per super-step
    int max_ss;
    double tol;           // relative residual stop, 0 = fixed count
    double tau_unit;      // tau_frac * 2 / lambda_max (mu~_j tau = mu_j * tau_unit)
    int* ss_done;         // device int
};
template <typename T>
size_t coarse_smem_bytes(long long n);
template <typename T>
bool coarse_fits(long long n);
template <typename T>
cudaError_t launch_coarse_solve(const CoarseParams& p, cudaStream_t st);
// Raise the dynamic shared-memory limit of the coarse kernels (once per process).
cudaError_t coarse_configure();

// ---- the two coarsest levels in one cluster launch (kernels_cluster.cu) ------
constexpr int kBottomMaxS = 32;          // smoothing stages the coefficient table holds
struct BottomParams {
    int nx, ny, nz;                      // level B; level C = B + 1 has half of each
    int per[3];                          // periodic flag per axis
    float hx, hy, hz;                    // 1 / h^2 of level B
    float chx, chy, chz;                 // 1 / h^2 of level C
    int order, s, n_pre, n_post;         // smoothing of level B
    float tau, mut1;                     // first stage: z = tau (L Y0 - f), Y1 = Y0 + mut1 z
    float mu[kBottomMaxS + 1], nu[kBottomMaxS + 1], mut_tau[kBottomMaxS + 1];
    float c0[kBottomMaxS + 1], gt[kBottomMaxS + 1];
    int remove_mean;                     // every axis periodic: f_C -= mean(f_C)
    const int* sched;                    // coarse solve: s per super-step (device)
    int max_ss;
    float tol;                           // relative residual stop, 0 = fixed count
    float tau_unit;                      // coarse: mu~_j tau = mu_j * tau_unit
    const float* rhs;                    // f_B (device)
    float* u_out;                        // e_B (device)
    int* ss_done;                        // coarse super-steps done (device int)
};
cudaError_t bottom_configure();
// Cluster size (0: not possible), block size and shared memory for level B.
int bottom_plan(int nx, int ny, int nz, int s, int* threads, size_t* bytes);
cudaError_t launch_bottom(const BottomParams& p, int nc, int threads, size_t bytes, cudaStream_t st);

}  // namespace sg
