// Host orchestration and C ABI (include/sg.h) of the RKL-multigrid solver.
//
// The grid owns per-level device buffers; a solve enqueues the V-cycle of
// Sec. 2.1 (smooth, residual + restrict, ..., coarsest RKL solve, prolong +
// correct, smooth) on the grid's stream, optionally captured once as a CUDA
// graph and replayed per cycle, and reads back one residual norm per cycle.
// In SG_MIXED the V-cycle runs in FP32 on the error equation L e = r, between
// an FP64 residual r = f - L phi and an FP64 update phi += e (defect
// correction); in SG_FP64 it runs in FP64 on phi directly.
#include "sg.h"
#include "sg_field_ops.cuh"
#include "sg_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

using namespace sg;

namespace {

thread_local std::string g_err;

sg_status fail(sg_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define SG_CK(...)                                                                               \
    do {                                                                                         \
        cudaError_t e_ = (__VA_ARGS__);                                                          \
        if (e_ != cudaSuccess)                                                                   \
            return fail(e_ == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA,              \
                        std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));              \
    } while (0)

#define SG_TRY(expr)                                                                             \
    do {                                                                                         \
        sg_status s_ = (expr);                                                                   \
        if (s_ != SG_OK) return s_;                                                              \
    } while (0)

struct Level {
    int nx = 0, ny = 0, nz = 0;
    long long n = 0;
    double h[3] = {0, 0, 0};
    void* u = nullptr;      // owned working-precision arrays (level 0 in FP64 mode: unused)
    void* rhs = nullptr;
    void* z0 = nullptr;
    void* t[3] = {nullptr, nullptr, nullptr};
};

// Stage coefficients of App. A (RKL1) and of the RKL2 member of the
// a_s + b_s P_s family (Meyer et al. 2014's b_j), written out here for the
// device path.
struct Rkl {
    int order, s;
    double w1, tau_over_dtpar;
    std::vector<double> mu, nu, mut, gt, c0;
};

Rkl make_rkl(int order, int s) {
    Rkl r;
    r.order = order;
    r.s = s;
    r.mu.assign(s + 1, 0.0);
    r.nu.assign(s + 1, 0.0);
    r.mut.assign(s + 1, 0.0);
    r.gt.assign(s + 1, 0.0);
    r.c0.assign(s + 1, 0.0);
    if (order == 1) {
        r.w1 = 2.0 / (double(s) * s + s);
        r.tau_over_dtpar = (double(s) * s + s) / 2.0;
        for (int j = 1; j <= s; ++j) {
            r.mu[j] = (2.0 * j - 1.0) / j;
            r.nu[j] = (1.0 - j) / j;
            r.mut[j] = r.mu[j] * r.w1;
        }
    } else {
        r.w1 = 4.0 / (double(s) * s + s - 2.0);
        r.tau_over_dtpar = (double(s) * s + s - 2.0) / 4.0;
        std::vector<double> b(s + 1), a(s + 1);
        for (int j = 0; j <= s; ++j) {
            b[j] = j <= 2 ? 1.0 / 3.0 : (double(j) * j + j - 2.0) / (2.0 * j * (j + 1.0));
            a[j] = 1.0 - b[j];
        }
        r.mut[1] = b[1] * r.w1;
        for (int j = 2; j <= s; ++j) {
            r.mu[j] = (2.0 * j - 1.0) / j * b[j] / b[j - 1];
            r.nu[j] = -(j - 1.0) / j * b[j] / b[j - 2];
            r.mut[j] = r.mu[j] * r.w1;
            r.gt[j] = -a[j - 1] * r.mut[j];
            r.c0[j] = 1.0 - r.mu[j] - r.nu[j];
        }
    }
    return r;
}

// Amplification of one super-step on the scalar test equation y' = -lambda y
// with tau = tau_frac * tau_max and lambda = lambda_max (the checkerboard
// mode), by the stage recurrence the kernels run: tau lambda_max = 2 tau_max /
// dt_par, so z = -2 tau_frac tau_max / dt_par.
double rkl_top_amplification(const Rkl& r, double tau_frac) {
    const double z = -2.0 * tau_frac * r.tau_over_dtpar;
    double y0 = 1.0, ym2 = 1.0, ym1 = 1.0 + r.mut[1] * z;
    for (int j = 2; j <= r.s; ++j) {
        const double y = r.mu[j] * ym1 + r.nu[j] * ym2 + r.c0[j] * y0 + (r.mut[j] * ym1 + r.gt[j] * y0) * z;
        ym2 = ym1;
        ym1 = y;
    }
    return ym1;
}

// Eq. sk_optimal: s_k = Round(2.4048 / pi * N / k - 1/2), halves rounded up.
int sk_opt(int k, int N) {
    const double p = 2.4048 / M_PI * (double(N) / double(k)) - 0.5;
    return (int)std::floor(p + 0.5);
}

// App. A.5 schedule that skips a k whose s repeats, k = N/2 .. 1, then s_1.
std::vector<int> accelerated_schedule(int N, int count) {
    std::vector<int> out;
    int k = std::max(1, N / 2);
    int s_old = 0;
    while ((int)out.size() < count) {
        const int s = std::max(1, sk_opt(k, N));
        if (!(s == s_old && k != 1)) {
            out.push_back(s);
            s_old = s;
        }
        k -= 1;
        if (k < 1) k = 1;
    }
    return out;
}

// P_s(x) by the three-term recursion of the Legendre polynomials.
double legendre_p(int s, double x) {
    if (s == 0) return 1.0;
    double pm = 1.0, p = x;
    for (int j = 2; j <= s; ++j) {
        const double pn = ((2.0 * j - 1.0) * x * p - (j - 1.0) * pm) / j;
        pm = p;
        p = pn;
    }
    return p;
}

// App. A.4: the first s at which lambda_k,RKL(s) = P_s(cos(k pi / N)) (Eq.
// eigenvalue_RKL) reaches zero or changes sign.
int first_zero_s(int k, int N) {
    const double x = std::cos(k * M_PI / N);
    double prev = 1.0;
    for (int s = 1;; ++s) {
        const double cur = legendre_p(s, x);
        if (cur == 0.0 || (cur > 0.0) != (prev > 0.0)) return s;
        prev = cur;
    }
}

// Eq. spectral_rad_RKL with k restricted to 1 .. min(6, N/2) (App. A.4, step 1).
double spectral_radius6(int s, int N) {
    const int kmax = std::min(6, std::max(1, N / 2));
    double r = 0.0;
    for (int k = 1; k <= kmax; ++k) r = std::max(r, std::fabs(legendre_p(s, std::cos(k * M_PI / N))));
    return r;
}

// App. A.4's two-step search for the single fixed s: the s in [first zero of
// lambda_1,RKL(s), N] with the smallest six-mode spectral radius (the first
// one on ties).
int s_opt_global(int N) {
    const int s0 = first_zero_s(1, N);
    int best = s0;
    double best_r = INFINITY;
    for (int s = s0; s <= std::max(s0, N); ++s) {
        const double r = spectral_radius6(s, N);
        if (r < best_r) {
            best_r = r;
            best = s;
        }
    }
    return best;
}

double cell_tau_frac(int N) {
    const double c = std::cos(M_PI / (2.0 * N));
    return c * c;
}

// Sec. 4.1's level rule on the x and y axes of a two-dimensional grid.
int rule_levels_2d(int nx, int ny) {
    int L = 1;
    auto ok = [](int n, int L) {
        const long long p = 1LL << L;
        return (n % p == 0) && ((n / p) % 2 == 0);
    };
    while (L < 30 && ok(nx, L) && ok(ny, L)) ++L;
    return L;
}

int rule_levels(int nx, int ny, int nz) {
    int L = 1;
    auto ok = [](int n, int L) {
        const long long p = 1LL << L;
        return (n % p == 0) && ((n / p) % 2 == 0);
    };
    while (L < 30 && ok(nx, L) && ok(ny, L) && ok(nz, L)) ++L;
    return L;
}

// Kernel classes for the optional per-kernel CUDA-event profile.
enum KClass { K_STAGE0 = 0, K_STAGE_C, K_RES0, K_RESTRICT, K_PROLONG, K_COARSE, K_UPDATE, K_MISC, K_BOTTOM,
              K_GSRB, K_GRAVITY, K_NCLASS };
const char* const kClassName[K_NCLASS] = {"rkl_stage_l0", "rkl_stage_coarse", "residual_l0",
                                          "residual_restrict", "prolong_correct", "coarse_solve",
                                          "update_residual", "reduce_misc", "bottom_levels",
                                          "gsrb_sweep", "gravity"};

struct ProfRec {
    int cls;
    double bytes;
    cudaEvent_t a, b;
};

}  // namespace

constexpr int kGraphKeySlots = 21;   // items the cached cycle graph is keyed on (run_cycle)

struct sg_grid {
    int n[3];
    bool twod = false;              // a two-dimensional grid (sg_create_grid_2d): nz = 1, no z term
    double lo[3], hi[3];
    int bc[3];
    int precision;
    cudaStream_t st;
    cudaStream_t own_stream = nullptr;
    int max_levels;
    std::vector<Level> lv;
    double* phi = nullptr;
    double* f = nullptr;
    double* faces[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool have_faces = false;
    double* gphi = nullptr;         // sg_gravity: a host potential, staged
    double* gout = nullptr;         // sg_gravity: the three components, staged for the host
    double* lam = nullptr;          // adjoint solution
    double* w = nullptr;            // adjoint source
    double* r64 = nullptr;          // FP64 residual f - A phi carried by recurrence (mixed)
    Partial* partials = nullptr;
    int partial_cap = 0;
    Reduced* red = nullptr;         // device slots
    Reduced* host_red = nullptr;    // pinned mirror
    int* d_sched = nullptr;
    int sched_cap = 0;
    int* d_ss = nullptr;            // coarse super-steps done (device)
    unsigned* d_mexp = nullptr;     // the exact residual's fixed-point scale (device)
    int* host_ss = nullptr;         // pinned mirror
    sg_options opt;
    double four_pi_G = 1.0;
    bool have_density = false;
    bool have_solution = false;
    bool guess_set = false;
    int last_levels = 0;
    // the cycle loop on the device: state (device and pinned mirror), the whole
    // solve as one graph (WHILE nodes), its key, and a serial number that
    // distinguishes grids created at a reused address
    DeviceLoop* dloop = nullptr;
    DeviceLoop* host_loop = nullptr;
    cudaGraphExec_t sexec = nullptr;
    uint64_t skey[kGraphKeySlots] = {0};
    long long s_per_cycle = 0, s_per_confirm = 0;   // kernels of one cycle / one confirmation in it
    unsigned long long serial = 0;
    // graph cache
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey[kGraphKeySlots] = {0};
    long long graph_launches = 0;
    long long launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // optional per-kernel profile
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<ProfRec> live;        // records of work enqueued outside a graph
    std::vector<ProfRec> graph_recs;  // records captured into the cached graph
    bool capturing = false;
    sg_kernel_stat stats[K_NCLASS];
};

namespace {

// Smoothing super-steps of level l on the way down / up: N_pre / N_post on
// level 0, the inner counts (when set) on levels 1 .. L-2.
int pre_count(const sg_grid* g, int l) {
    return (l > 0 && g->opt.inner_n_pre >= 0) ? g->opt.inner_n_pre : g->opt.n_pre;
}
int post_count(const sg_grid* g, int l) {
    return (l > 0 && g->opt.inner_n_post >= 0) ? g->opt.inner_n_post : g->opt.n_post;
}

bool all_periodic(const sg_grid* g) {
    return g->bc[0] == SG_BC_PERIODIC && g->bc[1] == SG_BC_PERIODIC && g->bc[2] == SG_BC_PERIODIC;
}

LevelGeom geom(const sg_grid* g, int l, bool with_faces) {
    const Level& L = g->lv[l];
    LevelGeom G;
    G.nx = L.nx;
    G.ny = L.ny;
    G.nz = L.nz;
    G.ihx2 = 1.0 / (L.h[0] * L.h[0]);
    G.ihy2 = 1.0 / (L.h[1] * L.h[1]);
    G.ihz2 = 1.0 / (L.h[2] * L.h[2]);
    G.ihx2f = float(G.ihx2);
    G.ihy2f = float(G.ihy2);
    G.ihz2f = float(G.ihz2);
    for (int d = 0; d < 3; ++d) G.per[d] = g->bc[d] == SG_BC_PERIODIC;
    for (int f = 0; f < 6; ++f) {
        const int d = f / 2;
        G.face[f] = (with_faces && l == 0 && g->bc[d] == SG_BC_DIRICHLET) ? g->faces[f] : nullptr;
    }
    G.twod = g->twod ? 1 : 0;
    return G;
}

double lambda_max(const Level& L) {
    return 4.0 * (1.0 / (L.h[0] * L.h[0]) + 1.0 / (L.h[1] * L.h[1]) + 1.0 / (L.h[2] * L.h[2]));
}

size_t wsize(const sg_grid* g) { return g->precision == SG_MIXED ? sizeof(float) : sizeof(double); }

cudaEvent_t take_event(sg_grid* g) {
    if (!g->ev_pool.empty()) {
        cudaEvent_t e = g->ev_pool.back();
        g->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one launch with CUDA events when profiling is on; `bytes` is the
// launch's algorithmic traffic (compulsory reads + writes of its arrays).
struct ProfScope {
    sg_grid* g;
    ProfRec rec;
    bool on;
    // During stream capture an event record must be marked external to become
    // an event node of the graph (outside capture the flag is not allowed).
    void record(cudaEvent_t e) {
        if (g->capturing) cudaEventRecordWithFlags(e, g->st, cudaEventRecordExternal);
        else cudaEventRecord(e, g->st);
    }
    ProfScope(sg_grid* g_, int cls, double bytes) : g(g_), on(g_->prof) {
        if (!on) return;
        rec.cls = cls;
        rec.bytes = bytes;
        rec.a = take_event(g);
        rec.b = take_event(g);
        record(rec.a);
    }
    ~ProfScope() {
        if (!on) return;
        record(rec.b);
        g->live.push_back(rec);
    }
};

// Fold completed records into the totals (the stream has been synchronised).
void prof_accumulate(sg_grid* g, std::vector<ProfRec>& recs, bool release) {
    for (const ProfRec& r : recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g->stats[r.cls].launches += 1;
            g->stats[r.cls].ms += ms;
            g->stats[r.cls].bytes += r.bytes;
        } else {
            cudaGetLastError();
        }
        if (release) {
            g->ev_pool.push_back(r.a);
            g->ev_pool.push_back(r.b);
        }
    }
    if (release) recs.clear();
}

void prof_sync_point(sg_grid* g, bool graph_replayed) {
    if (!g->prof) return;
    if (graph_replayed) prof_accumulate(g, g->graph_recs, false);
    prof_accumulate(g, g->live, true);
}

// Cap on cycles (single-level sweeps run tens of thousands); the info keeps
// the first SG_MAX_HISTORY residuals.
constexpr int kMaxCycles = 10000000;

sg_status check_opts(const sg_options* o) {
    if (o->rkl_order != 1 && o->rkl_order != 2) return fail(SG_ERR_ARG, "rkl_order must be 1 or 2");
    if (o->s_smooth < 1 || (o->rkl_order == 2 && o->s_smooth < 2) || o->s_smooth > 512)
        return fail(SG_ERR_ARG, "s_smooth out of range (RKL1: 1..512, RKL2: 2..512)");
    if (!(o->tau_frac > 0.0 && o->tau_frac <= 1.0)) return fail(SG_ERR_ARG, "tau_frac must be in (0, 1]");
    if (o->n_pre < 0 || o->n_post < 0 || o->n_pre + o->n_post < 1 || o->n_pre > 64 || o->n_post > 64)
        return fail(SG_ERR_ARG, "n_pre / n_post out of range");
    if (!(o->coarse_tol >= 0.0 && o->coarse_tol < 1.0)) return fail(SG_ERR_ARG, "coarse_tol must be in [0, 1)");
    if (o->coarse_max_ss < 1 || o->coarse_max_ss > 100000) return fail(SG_ERR_ARG, "coarse_max_ss out of range");
    if (!(o->coarse_tau_frac >= 0.0 && o->coarse_tau_frac <= 1.0)) return fail(SG_ERR_ARG, "coarse_tau_frac out of range");
    if (o->max_cycles < 1 || o->max_cycles > kMaxCycles) return fail(SG_ERR_ARG, "max_cycles out of range");
    if (o->single_s < -1 || o->single_s > 100000) return fail(SG_ERR_ARG, "single_s out of range");
    if (!(o->single_tau_frac >= 0.0 && o->single_tau_frac <= 1.0)) return fail(SG_ERR_ARG, "single_tau_frac out of range");
    if (o->fixed_cycles < 0 || o->fixed_cycles > kMaxCycles) return fail(SG_ERR_ARG, "fixed_cycles out of range");
    if (o->smoother != SG_SMOOTH_RKL && o->smoother != SG_SMOOTH_GSRB) return fail(SG_ERR_ARG, "unknown smoother");
    if (!(o->omega >= 0.0 && o->omega < 2.0)) return fail(SG_ERR_ARG, "omega must be in [0, 2)");
    if (!(o->max_residual_tol >= 0.0 && o->max_residual_tol < 1e300))
        return fail(SG_ERR_ARG, "max_residual_tol must be finite and >= 0");
    if (o->tile_rows != 0 && o->tile_rows != 14 && o->tile_rows != 16)
        return fail(SG_ERR_ARG, "tile_rows must be 0, 14 or 16");
    if (o->staging != SG_STAGE_CP_ASYNC && o->staging != SG_STAGE_TMA) return fail(SG_ERR_ARG, "unknown staging");
    if (o->host_copy != SG_HOST_COPY_ENGINE && o->host_copy != SG_HOST_COPY_KERNEL)
        return fail(SG_ERR_ARG, "unknown host_copy");
    if (o->use_graph < 0 || o->use_graph > 2) return fail(SG_ERR_ARG, "use_graph must be 0, 1 or 2");
    if (o->inner_n_pre < -1 || o->inner_n_pre > 64 || o->inner_n_post < -1 || o->inner_n_post > 64)
        return fail(SG_ERR_ARG, "inner_n_pre / inner_n_post out of range (-1 .. 64)");
    return SG_OK;
}

sg_status ensure_sched(sg_grid* g, const std::vector<int>& s) {
    if ((int)s.size() > g->sched_cap) {
        if (g->d_sched) cudaFree(g->d_sched);
        g->d_sched = nullptr;
        SG_CK(cudaMalloc(&g->d_sched, s.size() * sizeof(int)));
        g->sched_cap = (int)s.size();
    }
    SG_CK(cudaMemcpyAsync(g->d_sched, s.data(), s.size() * sizeof(int), cudaMemcpyHostToDevice, g->st));
    SG_CK(cudaStreamSynchronize(g->st));
    return SG_OK;
}

// ---- one RKL super-step at level l: u <- Y_s ---------------------------------
template <typename W>
sg_status superstep(sg_grid* g, int l, int order, int s, double tau_frac, bool faces, W* u,
                    const W* rhs) {
    const Level& L = g->lv[l];
    const LevelGeom G = geom(g, l, faces);
    const Rkl r = make_rkl(order, s);
    const double dtpar = 2.0 / lambda_max(L);
    const double tau = tau_frac * dtpar * r.tau_over_dtpar;
    W* t[3] = {(W*)L.t[0], (W*)L.t[1], (W*)L.t[2]};
    W* z0 = (W*)L.z0;
    StageCoef c{};
    c.tau = tau;
    c.mut1 = r.mut[1];
    W* out1 = t[0];
    const int cls = l == 0 ? K_STAGE0 : K_STAGE_C;
    const double nb = double(L.n) * sizeof(W);
    {
        ProfScope ps(g, cls, nb * (order == 2 ? 4 : 3));
        SG_CK(launch_stage<W>(G, order, true, c, u, nullptr, nullptr, nullptr, rhs, out1,
                              order == 2 ? z0 : nullptr, g->st));
    }
    ++g->launches;
    if (s == 1) {
        SG_CK(cudaMemcpyAsync(u, out1, L.n * sizeof(W), cudaMemcpyDeviceToDevice, g->st));
        return SG_OK;
    }
    for (int j = 2; j <= s; ++j) {
        StageCoef cj{};
        cj.mu = r.mu[j];
        cj.nu = r.nu[j];
        cj.mut_tau = r.mut[j] * tau;
        cj.c0 = r.c0[j];
        cj.gt = r.gt[j];
        const W* ym1 = (j - 1 == 0) ? u : t[(j - 2) % 3];
        const W* ym2 = (j - 2 == 0) ? u : t[(j - 3) % 3];
        W* out = (j == s) ? u : t[(j - 1) % 3];
        {
            ProfScope ps(g, cls, nb * (order == 2 ? 6 : 4));
            SG_CK(launch_stage<W>(G, order, false, cj, ym1, ym2, u, z0, rhs, out, nullptr, g->st));
        }
        ++g->launches;
    }
    return SG_OK;
}

// App. B: SOR omega = 2 / (1 + sqrt(1 - rho_J^2)) with the Jacobi radius
// rho_J = 2 dt sum_d cos(pi / n_d) / h_d^2, dt = (2 sum_d 1 / h_d^2)^-1 (the
// printed dt read as the inverse of the whole bracket, which gives the
// textbook Jacobi radius of a uniform cube).
double sor_omega(const Level& L) {
    const int n3[3] = {L.nx, L.ny, L.nz};
    double num = 0.0, den = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double ih2 = 1.0 / (L.h[d] * L.h[d]);
        num += std::cos(M_PI / n3[d]) * ih2;
        den += ih2;
    }
    const double rj = num / den;
    return 2.0 / (1.0 + std::sqrt(1.0 - rj * rj));
}

double gsrb_omega(const sg_grid* g, int l) {
    return g->opt.omega > 0.0 ? g->opt.omega : sor_omega(g->lv[l]);
}

// One red-black Gauss-Seidel / SOR sweep at level l (Sec. 2.2.4): the even
// cells, then the odd ones, each in place.
template <typename W>
sg_status gsrb_sweep(sg_grid* g, int l, bool faces, W* u, const W* rhs, double omega) {
    const LevelGeom G = geom(g, l, faces && l == 0);
    for (int colour = 0; colour < 2; ++colour) {
        {
            ProfScope ps(g, K_GSRB, 2.0 * g->lv[l].n * sizeof(W));
            SG_CK(launch_gsrb<W>(G, colour, omega, u, rhs, g->st));
        }
        ++g->launches;
    }
    return SG_OK;
}

template <typename W>
sg_status relax(sg_grid* g, int l, int count, bool faces, W* u, const W* rhs) {
    if (g->opt.smoother == SG_SMOOTH_GSRB) {
        const double om = gsrb_omega(g, l);
        for (int c = 0; c < count; ++c) SG_TRY(gsrb_sweep<W>(g, l, faces, u, rhs, om));
        return SG_OK;
    }
    for (int c = 0; c < count; ++c)
        SG_TRY(superstep<W>(g, l, g->opt.rkl_order, g->opt.s_smooth, g->opt.tau_frac, faces, u, rhs));
    return SG_OK;
}

double coarse_c(const sg_grid* g, int l) {
    const Level& L = g->lv[l];
    const int N = std::max(L.nx, std::max(L.ny, L.nz));
    return g->opt.coarse_tau_frac > 0.0 ? g->opt.coarse_tau_frac : cell_tau_frac(N);
}

// Coarsest-level solve of L u = rhs from u = 0 (homogeneous ghosts).
template <typename W>
sg_status coarse_solve(sg_grid* g, int l, const W* rhs, W* u, int* d_done) {
    const Level& L = g->lv[l];
    const int N = std::max(L.nx, std::max(L.ny, L.nz));
    if (coarse_fits<W>(L.n)) {
        CoarseParams p;
        p.g = geom(g, l, false);
        p.rhs = rhs;
        p.u_out = u;
        p.sched = g->d_sched;
        p.max_ss = g->opt.coarse_max_ss;
        p.tol = g->opt.coarse_tol;
        p.tau_unit = coarse_c(g, l) * 2.0 / lambda_max(L);
        p.ss_done = d_done;
        {
            ProfScope ps(g, K_COARSE, 2.0 * L.n * sizeof(W));
            SG_CK(launch_coarse_solve<W>(p, g->st));
        }
        ++g->launches;
        return SG_OK;
    }
    // Level too large for one CTA: stage kernels in global memory.
    const std::vector<int> sched = accelerated_schedule(N, g->opt.coarse_max_ss);
    SG_CK(cudaMemsetAsync(u, 0, L.n * sizeof(W), g->st));
    double r0 = -1.0;
    int done = 0;
    for (int ss = 0; ss < g->opt.coarse_max_ss; ++ss) {
        if (g->opt.coarse_tol > 0.0) {
            int nb = 0;
            SG_CK(launch_residual<W, W>(geom(g, l, false), u, rhs, (W*)nullptr, g->partials, &nb, g->st));
            SG_CK(launch_finalize(g->partials, nb, g->red + 3, g->st));
            SG_CK(cudaMemcpyAsync(g->host_red + 3, g->red + 3, sizeof(Reduced), cudaMemcpyDeviceToHost, g->st));
            SG_CK(cudaStreamSynchronize(g->st));
            g->launches += 2;
            const double rn = std::sqrt(g->host_red[3].sumsq);
            if (r0 < 0) r0 = rn;
            if (rn <= g->opt.coarse_tol * r0) break;
        }
        SG_TRY(superstep<W>(g, l, 1, sched[ss], coarse_c(g, l), false, u, rhs));
        ++done;
    }
    SG_CK(cudaMemcpyAsync(d_done, &done, sizeof(int), cudaMemcpyHostToDevice, g->st));
    SG_CK(cudaStreamSynchronize(g->st));
    return SG_OK;
}

// One fused super-step (FP32, homogeneous or periodic ghosts): out = Y_s(y0),
// y0 == nullptr meaning Y0 = 0.
sg_status superstep_fused(sg_grid* g, int l, int order, int s, double tau_frac, const float* y0,
                          const float* rhs, float* out) {
    const Level& L = g->lv[l];
    const Rkl r = make_rkl(order, s);
    const double tau = tau_frac * (2.0 / lambda_max(L)) * r.tau_over_dtpar;
    FusedCoef cf{};
    cf.tau = float(tau);
    cf.mut1 = float(r.mut[1]);
    for (int j = 2; j <= s; ++j) {
        cf.mu[j] = float(r.mu[j]);
        cf.nu[j] = float(r.nu[j]);
        cf.mut_tau[j] = float(r.mut[j] * tau);
        cf.c0[j] = float(r.c0[j]);
        cf.gt[j] = float(r.gt[j]);
    }
    {
        ProfScope ps(g, l == 0 ? K_STAGE0 : K_STAGE_C, double(L.n) * sizeof(float) * (y0 ? 3 : 2));
        SG_CK(launch_superstep_fused(geom(g, l, false), order, s, y0 == nullptr, cf, y0, rhs, out, g->st,
                                     g->opt.tile_rows, g->opt.staging == SG_STAGE_TMA));
    }
    ++g->launches;
    return SG_OK;
}

// The fused super-step streams each tile through all s stages one plane at a
// time; on small levels that serial chain of planes (its pipeline fill on
// short z chunks) costs more than it saves in HBM traffic (the level is
// L2-resident anyway), so only levels with at least kFusedMinCells cells use
// it: with the strip stage kernel, 128^3 runs faster as one launch per stage
// (7.72 against 7.85 ms per 256^3 solve).
constexpr long long kFusedMinCells = 1LL << 22;

bool use_fused(const sg_grid* g, bool faces, int l) {
    return !g->twod && g->precision == SG_MIXED && g->opt.fused && !faces && g->opt.smoother == SG_SMOOTH_RKL &&
           fused_supported(g->opt.rkl_order, g->opt.s_smooth) &&
           g->lv[l].n >= kFusedMinCells;
}

// The first super-step of a level's pre-smoothing starts from Y0 = 0: for
// s = 2, 3 the fused kernel runs it as s - 1 stencil stages of f in one launch,
// which beats s stage launches down to levels of kZeroFusedMinCells cells.
constexpr long long kZeroFusedMinCells = 1LL << 17;

bool use_fused_zero(const sg_grid* g, bool faces, int l) {
    return !g->twod && g->precision == SG_MIXED && g->opt.fused && !faces && g->opt.smoother == SG_SMOOTH_RKL &&
           g->opt.s_smooth <= 3 &&
           fused_supported(g->opt.rkl_order, g->opt.s_smooth) && g->lv[l].n >= kZeroFusedMinCells;
}

// The two coarsest levels B = L - 2 >= 1 and C = L - 1 of the FP32 V-cycle
// in one cluster launch (kernels_cluster.cu): the cluster size, or 0 where the
// level-by-level kernels run them.
int bottom_nc(const sg_grid* g, int L, int* threads, size_t* bytes) {
    const int B = L - 2;
    if (g->twod || g->precision != SG_MIXED || !g->opt.fused || g->opt.smoother != SG_SMOOTH_RKL || B < 1) return 0;
    const Level& lb = g->lv[B];
    return bottom_plan(lb.nx, lb.ny, lb.nz, g->opt.s_smooth, threads, bytes);
}

// e_B from f_B: B's pre-smoothing, the restriction to C, C's coarse solve, the
// prolongation to B and B's post-smoothing, with the coefficients and the
// schedule of the level-by-level path.
sg_status bottom_levels(sg_grid* g, int B, const float* rhs, float* u, int nc, int threads, size_t bytes) {
    const Level& lb = g->lv[B];
    const Level& lc = g->lv[B + 1];
    const LevelGeom gb = geom(g, B, false), gc = geom(g, B + 1, false);
    const int order = g->opt.rkl_order, s = g->opt.s_smooth;
    const Rkl r = make_rkl(order, s);
    const double tau = g->opt.tau_frac * (2.0 / lambda_max(lb)) * r.tau_over_dtpar;
    BottomParams p{};
    p.nx = lb.nx;
    p.ny = lb.ny;
    p.nz = lb.nz;
    for (int d = 0; d < 3; ++d) p.per[d] = gb.per[d];
    p.hx = gb.ihx2f;
    p.hy = gb.ihy2f;
    p.hz = gb.ihz2f;
    p.chx = gc.ihx2f;
    p.chy = gc.ihy2f;
    p.chz = gc.ihz2f;
    p.order = order;
    p.s = s;
    p.n_pre = pre_count(g, B);
    p.n_post = post_count(g, B);
    p.tau = float(tau);
    p.mut1 = float(r.mut[1]);
    for (int j = 2; j <= s; ++j) {
        p.mu[j] = float(r.mu[j]);
        p.nu[j] = float(r.nu[j]);
        p.mut_tau[j] = float(r.mut[j] * tau);
        p.c0[j] = float(r.c0[j]);
        p.gt[j] = float(r.gt[j]);
    }
    p.remove_mean = all_periodic(g) ? 1 : 0;
    p.sched = g->d_sched;
    p.max_ss = g->opt.coarse_max_ss;
    p.tol = float(g->opt.coarse_tol);
    p.tau_unit = float(coarse_c(g, B + 1) * 2.0 / lambda_max(lc));
    p.rhs = rhs;
    p.u_out = u;
    p.ss_done = g->d_ss;
    {
        ProfScope ps(g, K_BOTTOM, 2.0 * lb.n * sizeof(float));
        SG_CK(launch_bottom(p, nc, threads, bytes, g->st));
    }
    ++g->launches;
    return SG_OK;
}

// One V-cycle (Sec. 2.1) with level-0 arrays u0 / rhs0 (faces on level 0 if
// `faces`; zero0: u0 is known to be zero, as for the error equation of the
// mixed-precision loop).  On return *u0_final points at the level-0 result: u0
// itself, or, with the fused FP32 super-steps (which cannot write in place),
// whichever of u0 and its ping-pong partner holds it.
template <typename W>
sg_status vcycle(sg_grid* g, int L, W* u0, const W* rhs0, bool faces, bool zero0, W** u0_final) {
    W* cur[32];
    W* alt[32];
    for (int l = 0; l < L; ++l) {
        cur[l] = l == 0 ? u0 : (W*)g->lv[l].u;
        alt[l] = (W*)g->lv[l].t[0];
    }
    auto R = [&](int l) -> const W* { return l == 0 ? rhs0 : (const W*)g->lv[l].rhs; };
    const bool per = all_periodic(g);
    // `count` smoothing super-steps at level l; zero_start: the level's u is 0.
    auto smooth = [&](int l, int count, bool zero_start, bool fc) -> sg_status {
        if constexpr (std::is_same<W, float>::value) {
            if (use_fused(g, fc, l)) {
                for (int c = 0; c < count; ++c) {
                    const bool z = zero_start && c == 0;
                    float* out = z ? cur[l] : alt[l];
                    SG_TRY(superstep_fused(g, l, g->opt.rkl_order, g->opt.s_smooth, g->opt.tau_frac,
                                           z ? nullptr : cur[l], R(l), out));
                    if (!z) std::swap(cur[l], alt[l]);
                }
                if (zero_start && count == 0) SG_CK(cudaMemsetAsync(cur[l], 0, g->lv[l].n * sizeof(W), g->st));
                return SG_OK;
            }
            if (zero_start && count > 0 && use_fused_zero(g, fc, l)) {
                SG_TRY(superstep_fused(g, l, g->opt.rkl_order, g->opt.s_smooth, g->opt.tau_frac, nullptr, R(l),
                                       cur[l]));
                return relax<W>(g, l, count - 1, fc, cur[l], R(l));
            }
        }
        if (zero_start) SG_CK(cudaMemsetAsync(cur[l], 0, g->lv[l].n * sizeof(W), g->st));   // also for count = 0
        return relax<W>(g, l, count, fc, cur[l], R(l));
    };
    int bottom_threads = 0;
    size_t bottom_bytes = 0;
    const int bottom = std::is_same<W, float>::value ? bottom_nc(g, L, &bottom_threads, &bottom_bytes) : 0;
    SG_TRY(smooth(0, g->opt.n_pre, zero0, faces));                              // step 1
    for (int l = 1; l < L; ++l) {                                               // step 2
        if (bottom && l == L - 1) break;        // restricted into C inside the cluster launch
        int nb = 0;
        {
            ProfScope ps(g, K_RESTRICT, (2.0 + 0.125) * g->lv[l - 1].n * sizeof(W));
            SG_CK(launch_residual_restrict<W>(geom(g, l - 1, faces && l - 1 == 0), cur[l - 1], R(l - 1),
                                              (W*)g->lv[l].rhs, g->partials, &nb, g->st));   // 2a, 2b
        }
        ++g->launches;
        if (per) {                                                              // coarse mean removed
            ProfScope ps(g, K_MISC, 2.0 * g->lv[l].n * sizeof(W));
            SG_CK(launch_finalize(g->partials, nb, g->red + 1, g->st));
            SG_CK(launch_subtract_mean<W>((W*)g->lv[l].rhs, g->lv[l].n, g->red + 1, g->st));
            g->launches += 2;
        }
        if constexpr (std::is_same<W, float>::value) {
            if (bottom && l == L - 2) {                                          // levels L - 2 and L - 1
                SG_TRY(bottom_levels(g, l, R(l), cur[l], bottom, bottom_threads, bottom_bytes));
                continue;
            }
        }
        if (l < L - 1) SG_TRY(smooth(l, pre_count(g, l), true, false));         // 2c + 2d-i
        else SG_TRY(coarse_solve<W>(g, l, R(l), cur[l], g->d_ss));              // 2c + 2e
    }
    for (int l = L - 2; l >= 1; --l) {                                          // step 3
        if (bottom && l == L - 2) continue;     // prolonged and post-smoothed in the cluster launch
        {
            ProfScope ps(g, K_PROLONG, (2.0 + 0.125) * g->lv[l].n * sizeof(W));
            SG_CK(launch_prolong_correct<W>(geom(g, l, false), cur[l + 1], cur[l], g->st));
        }
        ++g->launches;
        SG_TRY(smooth(l, post_count(g, l), false, false));
    }
    {
        ProfScope ps(g, K_PROLONG, (2.0 + 0.125) * g->lv[0].n * sizeof(W));
        SG_CK(launch_prolong_correct<W>(geom(g, 0, false), cur[1], cur[0], g->st));  // 4a
    }
    ++g->launches;
    SG_TRY(smooth(0, g->opt.n_post, false, faces));                             // 4b
    if (u0_final) *u0_final = cur[0];
    return SG_OK;
}

// Residual norm of (phi, f) at level 0 into red[0]; mixed mode also writes r32.
sg_status level0_residual(sg_grid* g, const double* phi, const double* f, bool faces) {
    int nb = 0, nk = 1;
    const LevelGeom G = geom(g, 0, faces);
    {
    ProfScope ps(g, K_RES0, double(g->lv[0].n) * (g->precision == SG_MIXED ? 28.0 : 16.0));
    if (g->precision == SG_MIXED)
        SG_CK(launch_residual_exact(G, phi, f, (float*)g->lv[0].rhs, g->r64, g->partials, g->d_mexp, &nb, &nk,
                                    g->st));
    else
        SG_CK(launch_residual<double, double>(G, phi, f, (double*)nullptr, g->partials, &nb, g->st));
    }
    SG_CK(launch_finalize(g->partials, nb, g->red, g->st));
    g->launches += nk + 1;
    return SG_OK;
}

// level0_residual for phi = 0 (no read of phi, no FP64 stencil).
sg_status level0_residual_zero(sg_grid* g, const double* f, bool faces) {
    int nb = 0, nk = 1;
    const LevelGeom G = geom(g, 0, faces);
    {
    ProfScope ps(g, K_RES0, double(g->lv[0].n) * (g->precision == SG_MIXED ? 20.0 : 8.0));
    if (g->precision == SG_MIXED)
        SG_CK(launch_residual_zero<float>(G, f, (float*)g->lv[0].rhs, g->partials, &nb, g->st, g->r64, &nk));
    else
        SG_CK(launch_residual_zero<double>(G, f, (double*)nullptr, g->partials, &nb, g->st, nullptr, &nk));
    }
    SG_CK(launch_finalize(g->partials, nb, g->red, g->st));
    g->launches += nk + 1;
    return SG_OK;
}

// Everything one cycle enqueues after the first residual: V-cycle, update,
// residual + norm, and the copies of the norm / coarse count to pinned memory.
// One V-cycle and the residual norm after it (into red[0]); no host copies.
sg_status cycle_core(sg_grid* g, int L, double* phi, const double* f, bool faces) {
    if (g->precision == SG_MIXED) {
        // the inner cycle starts from e = 0: its first super-step takes Y0 = 0
        float* e = (float*)g->lv[0].u;
        float* e_final = e;
        SG_TRY(vcycle<float>(g, L, e, (const float*)g->lv[0].rhs, false, true, &e_final));
        // phi += e and the FP64 residual by recurrence r -= A_0 e (and its FP32 copy)
        int nb = 0;
        {
            ProfScope ps(g, K_UPDATE, 40.0 * g->lv[0].n);
            SG_CK(launch_update_residual(geom(g, 0, false), phi, e_final, g->r64, (float*)g->lv[0].rhs,
                                         g->partials, &nb, g->st));
        }
        SG_CK(launch_finalize(g->partials, nb, g->red, g->st));
        g->launches += 2;
    } else {
        SG_TRY(vcycle<double>(g, L, phi, f, faces, false, nullptr));
        SG_TRY(level0_residual(g, phi, f, faces));
    }
    return SG_OK;
}

sg_status cycle_body(sg_grid* g, int L, double* phi, const double* f, bool faces) {
    SG_TRY(cycle_core(g, L, phi, f, faces));
    SG_CK(cudaMemcpyAsync(g->host_red, g->red, sizeof(Reduced), cudaMemcpyDeviceToHost, g->st));
    SG_CK(cudaMemcpyAsync(g->host_ss, g->d_ss, sizeof(int), cudaMemcpyDeviceToHost, g->st));
    return SG_OK;
}

void drop_graph(sg_grid* g) {
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
    if (g->sexec) cudaGraphExecDestroy(g->sexec);
    g->sexec = nullptr;
    std::memset(g->skey, 0, sizeof(g->skey));
    std::memset(g->gkey, 0, sizeof(g->gkey));
    for (const ProfRec& r : g->graph_recs) {
        g->ev_pool.push_back(r.a);
        g->ev_pool.push_back(r.b);
    }
    g->graph_recs.clear();
}

// Whether the V-cycle can be captured into a CUDA graph (the coarsest level
// fits one CTA: the larger coarse solve reads its norm on the host).
bool cycle_graphable(const sg_grid* g, int L) {
    return g->opt.use_graph && L > 1 &&
           (g->precision == SG_MIXED ? coarse_fits<float>(g->lv[L - 1].n) : coarse_fits<double>(g->lv[L - 1].n));
}

// Everything a captured cycle depends on, one slot per item (doubles by their
// bit pattern), compared slot by slot: no scaling, no folding.
void graph_key(const sg_grid* g, int L, const double* phi, const double* f, bool faces, uint64_t key[kGraphKeySlots]) {
    auto bits = [](double v) {
        uint64_t u;
        std::memcpy(&u, &v, sizeof(u));
        return u;
    };
    const uint64_t k[kGraphKeySlots] = {(uint64_t)L, (uint64_t)(uintptr_t)phi, (uint64_t)(uintptr_t)f,
                                        faces ? 1u : 0u, (uint64_t)g->opt.rkl_order, (uint64_t)g->opt.s_smooth,
                                        bits(g->opt.tau_frac), (uint64_t)g->opt.n_pre, (uint64_t)g->opt.n_post,
                                        bits(g->opt.coarse_tol), (uint64_t)g->opt.coarse_max_ss,
                                        bits(g->opt.coarse_tau_frac), (uint64_t)g->opt.smoother,
                                        bits(g->opt.omega), (uint64_t)(g->opt.fused ? 1 : 0),
                                        (uint64_t)(g->prof ? 1 : 0), (uint64_t)(uintptr_t)g->d_sched,
                                        (uint64_t)g->opt.tile_rows, (uint64_t)g->opt.staging,
                                        (uint64_t)(int64_t)g->opt.inner_n_pre, (uint64_t)(int64_t)g->opt.inner_n_post};
    std::memcpy(key, k, sizeof(k));
}

sg_status run_cycle(sg_grid* g, int L, double* phi, const double* f, bool faces, bool* replayed) {
    *replayed = false;
    if (!cycle_graphable(g, L)) return cycle_body(g, L, phi, f, faces);
    uint64_t key[kGraphKeySlots];
    graph_key(g, L, phi, f, faces, key);
    if (!g->gexec || std::memcmp(key, g->gkey, sizeof(key)) != 0) {
        drop_graph(g);
        cudaGraph_t graph = nullptr;
        const long long before = g->launches;
        SG_CK(cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal));
        std::vector<ProfRec> outside;
        outside.swap(g->live);
        g->capturing = true;
        sg_status s = cycle_body(g, L, phi, f, faces);
        g->capturing = false;
        cudaError_t ec = cudaStreamEndCapture(g->st, &graph);
        g->live.swap(outside);          // g->live: records enqueued before the capture
        if (s != SG_OK) {
            if (graph) cudaGraphDestroy(graph);
            for (const ProfRec& r : outside) { g->ev_pool.push_back(r.a); g->ev_pool.push_back(r.b); }
            return s;
        }
        if (ec != cudaSuccess) return fail(SG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
        cudaError_t ei = cudaGraphInstantiate(&g->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            g->gexec = nullptr;
            return fail(SG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
        }
        g->graph_launches = g->launches - before;
        g->launches = before;
        std::memcpy(g->gkey, key, sizeof(key));
        g->graph_recs.swap(outside);    // the records captured into the graph
    }
    SG_CK(cudaGraphLaunch(g->gexec, g->st));
    g->launches += g->graph_launches;
    *replayed = true;
    return SG_OK;
}

long long stage_updates_per_cycle(const sg_grid* g, int L) {
    long long su = 0;
    const int per_relax = g->opt.smoother == SG_SMOOTH_GSRB ? 1 : g->opt.s_smooth;   // a sweep updates a cell once
    for (int l = 0; l < L - 1; ++l)
        su += (long long)g->lv[l].n * (pre_count(g, l) + post_count(g, l)) * per_relax;
    return su;
}

// The solve loop shared by sg_solve (phi, f, faces) and sg_backward (lam, w, none).
// State of one solve between its set-up, its cycles and its wrap-up (shared by
// sg_solve and sg_solve_batch).
struct SolveState {
    sg_solve_info info;
    long long launches0 = 0;
    int L = 1;
    double* phi = nullptr;
    const double* f = nullptr;
    bool faces = false;
    double tol = 0.0;
    double nn = 1.0, rden = 1.0;
    int limit = 0;
    double single_c = 1.0;
    std::vector<int> single_sched;
    int single_s_opt = 0;           // single_s = -1: App. A.4's global s_opt of the level
    long long su = 0;
    int m = 0;
    bool done = false;
    sg_status status = SG_OK;
};

// r0 = ||L 0 - f|| (boundary contribution of phi = 0 included), the first
// residual, the coarse schedule; leaves the residual of the start in host_red[0].
sg_status solve_begin(sg_grid* g, SolveState& S, double tol, int L, double* phi, const double* f, bool faces,
                      bool have_guess) {
    if (g->opt.smoother == SG_SMOOTH_GSRB) {
        // red-black colouring must hold across a periodic wrap on every swept level
        for (int l = 0; l < std::max(1, L - 1); ++l) {
            const int n3[3] = {g->lv[l].nx, g->lv[l].ny, g->lv[l].nz};
            for (int d = 0; d < (g->twod ? 2 : 3); ++d)
                if (g->bc[d] == SG_BC_PERIODIC && (n3[d] & 1))
                    return fail(SG_ERR_ARG, "GS-RB smoothing needs even extents on periodic axes");
        }
    }
    std::memset(&S.info, 0, sizeof(S.info));
    S.info.levels = L;
    S.info.s_smooth = g->opt.s_smooth;
    S.info.rkl_order = g->opt.rkl_order;
    S.info.precision = g->precision;
    S.launches0 = g->launches;
    S.L = L;
    S.phi = phi;
    S.f = f;
    S.faces = faces;
    S.tol = tol;
    const Level& L0 = g->lv[0];
    SG_CK(cudaEventRecord(g->ev0, g->st));
    if (!have_guess) {
        SG_CK(cudaMemsetAsync(phi, 0, L0.n * sizeof(double), g->st));
        SG_TRY(level0_residual_zero(g, f, faces));
    } else {
        // r0 = ||L 0 - f|| for the relative stopping test, then the guess's residual
        SG_TRY(level0_residual_zero(g, f, faces));
        SG_CK(cudaMemcpyAsync(g->host_red + 2, g->red, sizeof(Reduced), cudaMemcpyDeviceToHost, g->st));
        SG_TRY(level0_residual(g, phi, f, faces));
    }
    SG_CK(cudaMemcpyAsync(g->host_red, g->red, sizeof(Reduced), cudaMemcpyDeviceToHost, g->st));
    SG_CK(cudaStreamSynchronize(g->st));
    prof_sync_point(g, false);
    S.nn = double(L0.n);
    const double r0 = std::sqrt((have_guess ? g->host_red[2].sumsq : g->host_red[0].sumsq) / S.nn);
    S.info.r0 = r0;
    S.rden = r0 > 0.0 ? r0 : 1.0;
    const int N0 = std::max(L0.nx, std::max(L0.ny, L0.nz));
    if (L == 1) {
        // every distinct entry: the schedule repeats its last value (k = 1) from there on
        S.single_sched = accelerated_schedule(N0, N0 / 2 + 2);
        S.single_s_opt = g->opt.single_s < 0 ? s_opt_global(N0) : 0;
    } else {
        const Level& Lc = g->lv[L - 1];
        const int Nc = std::max(Lc.nx, std::max(Lc.ny, Lc.nz));
        SG_TRY(ensure_sched(g, accelerated_schedule(Nc, g->opt.coarse_max_ss)));
        int bt = 0;
        size_t bb = 0;
        (void)bottom_nc(g, L, &bt, &bb);          // plan the cluster launch before any capture
    }
    S.limit = g->opt.fixed_cycles > 0 ? g->opt.fixed_cycles : g->opt.max_cycles;
    S.single_c = g->opt.single_tau_frac > 0 ? g->opt.single_tau_frac : cell_tau_frac(N0);
    S.su = 0;
    S.m = 0;
    S.done = false;
    S.status = SG_OK;
    return SG_OK;
}

// Record the residual now in host_red[0]; decide whether the solve is over.
// Mixed precision carries the FP64 residual by recurrence between cycles; when
// it reaches the tolerance, the true FP64 residual f - A phi is computed once to
// confirm (and, should it not confirm, the recurrence restarts from it).
sg_status solve_check(sg_grid* g, SolveState& S) {
    // the stopping test: relative L2 (Sec. 4.1) or, when max_residual_tol is
    // set, the maximum residual (App. B)
    const double mtol = g->opt.max_residual_tol;
    auto met = [&](double rel, double maxabs) { return mtol > 0.0 ? maxabs <= mtol : rel <= S.tol; };
    double rel = std::sqrt(g->host_red[0].sumsq / S.nn) / S.rden;
    if (g->opt.fixed_cycles == 0 && met(rel, g->host_red[0].maxabs) && std::isfinite(rel) &&
        g->precision == SG_MIXED && S.L > 1) {
        SG_TRY(level0_residual(g, S.phi, S.f, S.faces));
        SG_CK(cudaMemcpyAsync(g->host_red, g->red, sizeof(Reduced), cudaMemcpyDeviceToHost, g->st));
        SG_CK(cudaStreamSynchronize(g->st));
        prof_sync_point(g, false);
        rel = std::sqrt(g->host_red[0].sumsq / S.nn) / S.rden;
    }
    if (S.m < SG_MAX_HISTORY) S.info.history[S.m] = rel;
    S.info.rel_residual = rel;
    S.info.max_residual = g->host_red[0].maxabs;
    if (!std::isfinite(rel)) {
        const unsigned waits = g->precision == SG_MIXED ? lean_wait_failures() : 0u;
        S.status = fail(SG_ERR_NONFINITE, waits ? "residual norm is not finite: " + std::to_string(waits) +
                                                      " fused super-step launch(es) gave up a bounded wait"
                                                : std::string("residual norm is not finite"));
        S.done = true;
    } else if (g->opt.fixed_cycles == 0 && met(rel, g->host_red[0].maxabs)) {
        S.done = true;
    } else if (S.m >= S.limit) {
        if (g->opt.fixed_cycles == 0) S.status = fail(SG_ERR_NOT_CONVERGED, "max_cycles reached above the tolerance");
        S.done = true;
    }
    return SG_OK;
}

// One single-level super-step (levels == 1), its residual and norm copy.
sg_status solve_single_step(sg_grid* g, SolveState& S) {
    const Level& L0 = g->lv[0];
    if (g->opt.smoother == SG_SMOOTH_GSRB) {
        // one red-black Gauss-Seidel / SOR sweep (App. B); mixed precision sweeps
        // the error equation from e = 0, which gives the same correction
        const double om = gsrb_omega(g, 0);
        if (g->precision == SG_MIXED) {
            float* e = (float*)L0.u;
            SG_CK(cudaMemsetAsync(e, 0, L0.n * sizeof(float), g->st));
            SG_TRY(gsrb_sweep<float>(g, 0, false, e, (const float*)L0.rhs, om));
            {
                ProfScope ps(g, K_UPDATE, 20.0 * L0.n);
                SG_CK(launch_add_f32_to_f64(S.phi, e, L0.n, g->st));
            }
            ++g->launches;
        } else {
            SG_TRY(gsrb_sweep<double>(g, 0, S.faces, S.phi, S.f, om));
        }
        S.su += L0.n;
        SG_TRY(level0_residual(g, S.phi, S.f, S.faces));
        SG_CK(cudaMemcpyAsync(g->host_red, g->red, sizeof(Reduced), cudaMemcpyDeviceToHost, g->st));
        *g->host_ss = 0;
        return SG_OK;
    }
    const int s = g->opt.single_s > 0   ? g->opt.single_s
                  : g->opt.single_s < 0 ? S.single_s_opt
                                        : S.single_sched[std::min<size_t>(S.m, S.single_sched.size() - 1)];
    if (g->precision == SG_MIXED) {
        // mixed precision: an FP32 super-step on the error equation L e = r
        float* e = (float*)L0.u;
        SG_CK(cudaMemsetAsync(e, 0, L0.n * sizeof(float), g->st));
        SG_TRY(superstep<float>(g, 0, 1, s, S.single_c, false, e, (const float*)L0.rhs));
        {
            ProfScope ps(g, K_UPDATE, 20.0 * L0.n);
            SG_CK(launch_add_f32_to_f64(S.phi, e, L0.n, g->st));
        }
        ++g->launches;
    } else {
        SG_TRY(superstep<double>(g, 0, 1, s, S.single_c, S.faces, S.phi, S.f));
    }
    S.su += L0.n * (long long)s;
    SG_TRY(level0_residual(g, S.phi, S.f, S.faces));
    SG_CK(cudaMemcpyAsync(g->host_red, g->red, sizeof(Reduced), cudaMemcpyDeviceToHost, g->st));
    *g->host_ss = 0;
    return SG_OK;
}

// Book-keeping after a cycle's work has completed (stream synchronised).
void solve_after_cycle(sg_grid* g, SolveState& S) {
    if (S.L > 1) {
        S.su += stage_updates_per_cycle(g, S.L);
        if (S.m < SG_MAX_HISTORY) S.info.coarse_ss[S.m] = *g->host_ss;
        const Level& Lc = g->lv[S.L - 1];
        const int Nc = std::max(Lc.nx, std::max(Lc.ny, Lc.nz));
        const std::vector<int> sc = accelerated_schedule(Nc, std::max(1, *g->host_ss));
        for (int q = 0; q < *g->host_ss && q < (int)sc.size(); ++q) S.su += Lc.n * (long long)sc[q];
    }
    ++S.m;
}

sg_status solve_end(sg_grid* g, SolveState& S, sg_solve_info* info) {
    const Level& L0 = g->lv[0];
    S.info.cycles = S.m;
    if (all_periodic(g)) {
        int nb = 0;
        SG_CK(launch_sum_partials_f64(S.phi, L0.n, g->partials, &nb, g->st));
        SG_CK(launch_finalize(g->partials, nb, g->red + 1, g->st));
        SG_CK(launch_sub_mean_f64(S.phi, L0.n, g->red + 1, g->st));
        g->launches += 3;
    }
    SG_CK(cudaEventRecord(g->ev1, g->st));
    SG_CK(cudaEventSynchronize(g->ev1));
    float ms = 0.f;
    SG_CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    S.info.elapsed_ms = ms;
    S.info.stage_cell_updates = S.su;
    S.info.kernel_launches = g->launches - S.launches0;
    S.info.status = S.status;
    if (info) *info = S.info;
    return S.status;
}

// ---- the whole solve as one graph ------------------------------------------------
// Appends the cycle loop of grid g to `graph`, as a branch with no incoming
// edge (a batch adds one branch per grid):
//   init -> WHILE(outer) { WHILE(inner) { V-cycle, residual norm, step }
//                          [mixed: the true FP64 residual]  confirm }
// The one-thread init / step / confirm kernels (kernels_loop.cu) take the host
// loop's decisions on the device and set the two conditions.  *per_cycle and
// *per_confirm receive the kernels of one inner and one outer iteration.
sg_status add_solve_loop(sg_grid* g, cudaGraph_t graph, int L, double* phi, const double* f, bool faces,
                         long long* per_cycle, long long* per_confirm) {
    cudaStream_t st = g->st;
    cudaGraphConditionalHandle ho = 0, hi = 0;
    SG_CK(cudaGraphConditionalHandleCreate(&ho, graph, 0, cudaGraphCondAssignDefault));
    SG_CK(cudaGraphConditionalHandleCreate(&hi, graph, 0, cudaGraphCondAssignDefault));
    // appends a WHILE node after the work captured so far on st; returns its body
    auto add_while = [&](cudaGraphConditionalHandle h, cudaGraph_t* body) -> sg_status {
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        SG_CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &nd));
        // zero-initialised storage: the parameter union has no default constructor
        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};
        cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        SG_CK(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &cp));
        *body = cp.conditional.phGraph_out[0];
        SG_CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        return SG_OK;
    };
    // a capture into `target` that always ends, even on an error
    auto capture = [&](cudaGraph_t target, auto&& fill) -> sg_status {
        SG_CK(cudaStreamBeginCaptureToGraph(st, target, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        const sg_status s = fill();
        cudaGraph_t out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &out);
        if (s != SG_OK) return s;
        if (e != cudaSuccess) return fail(SG_ERR_CUDA, std::string("solve graph capture: ") + cudaGetErrorString(e));
        return SG_OK;
    };
    cudaGraph_t outer_body = nullptr, inner_body = nullptr;
    SG_TRY(capture(graph, [&]() -> sg_status {
        SG_CK(launch_loop_init(g->dloop, ho, hi, st));
        return add_while(ho, &outer_body);
    }));
    const long long before = g->launches;
    SG_TRY(capture(outer_body, [&]() -> sg_status {
        SG_TRY(add_while(hi, &inner_body));
        const long long b0 = g->launches;
        if (g->precision == SG_MIXED) SG_TRY(level0_residual(g, phi, f, faces));
        SG_CK(launch_loop_confirm(g->dloop, g->red, ho, hi, st));
        *per_confirm = g->launches - b0 + 1;
        return SG_OK;
    }));
    SG_TRY(capture(inner_body, [&]() -> sg_status {
        const long long b0 = g->launches;
        SG_TRY(cycle_core(g, L, phi, f, faces));
        SG_CK(launch_loop_step(g->dloop, g->red, g->d_ss, g->d_sched, hi, st));
        *per_cycle = g->launches - b0 + 1;
        return SG_OK;
    }));
    g->launches = before;
    return SG_OK;
}

// State of the device loop for the solve S (after the host's first check).
void fill_device_loop(sg_grid* g, const SolveState& S, DeviceLoop* d) {
    std::memset(d, 0, sizeof(*d));
    d->rden = S.rden;
    d->nn = S.nn;
    d->tol = S.tol;
    d->mtol = g->opt.max_residual_tol;
    d->limit = S.limit;
    d->fixed = g->opt.fixed_cycles > 0 ? 1 : 0;
    d->confirm = (g->precision == SG_MIXED && S.L > 1) ? 1 : 0;
    d->m = S.m;
    d->status = S.done ? kLoopDone : kLoopRunning;
    d->sched_len = g->opt.coarse_max_ss;
    const Level& Lc = g->lv[S.L - 1];
    d->coarse_cells = Lc.n;
    d->rel = S.info.rel_residual;
    d->maxabs = S.info.max_residual;
    d->history[0] = S.info.history[0];
}

// Results of a finished device loop into S.
void read_device_loop(sg_grid* g, SolveState& S, const DeviceLoop& d, long long per_cycle, long long per_confirm) {
    const int m0 = S.m;
    S.m = d.m;
    for (int q = m0 + 1; q <= d.m && q < SG_MAX_HISTORY; ++q) S.info.history[q] = d.history[q];
    for (int q = m0; q < d.m && q < SG_MAX_HISTORY; ++q) S.info.coarse_ss[q] = d.coarse_ss[q];
    S.info.rel_residual = d.rel;
    S.info.max_residual = d.maxabs;
    S.su += (long long)(d.m - m0) * stage_updates_per_cycle(g, S.L) + d.coarse_stage_cells;
    g->launches += 1 + (long long)(d.m - m0) * per_cycle + (long long)d.confirms * per_confirm;
    if (d.status == kLoopNonFinite) {
        const unsigned waits = g->precision == SG_MIXED ? lean_wait_failures() : 0u;
        S.status = fail(SG_ERR_NONFINITE, waits ? "residual norm is not finite: " + std::to_string(waits) +
                                                      " fused super-step launch(es) gave up a bounded wait"
                                                : std::string("residual norm is not finite"));
    } else if (d.status == kLoopNotConverged) {
        S.status = fail(SG_ERR_NOT_CONVERGED, "max_cycles reached above the tolerance");
    }
    S.done = true;
}

// Whether a solve runs as one graph with its cycle loop on the device: the
// cycle can be captured and no per-kernel profile is being taken (the
// profile's event records cannot sit inside a conditional body).
bool use_device_loop(const sg_grid* g, int L) {
    return g->opt.use_graph == 1 && cycle_graphable(g, L) && !g->prof && g->dloop != nullptr;
}

void drop_solve_graph(sg_grid* g) {
    if (g->sexec) cudaGraphExecDestroy(g->sexec);
    g->sexec = nullptr;
    std::memset(g->skey, 0, sizeof(g->skey));
}

// The cycles of solve S as one graph launch (captured once per key), the
// loop state written before and read back after it: one host round trip.
sg_status run_device_loop(sg_grid* g, SolveState& S) {
    uint64_t key[kGraphKeySlots];
    graph_key(g, S.L, S.phi, S.f, S.faces, key);
    if (!g->sexec || std::memcmp(key, g->skey, sizeof(key)) != 0) {
        drop_solve_graph(g);
        cudaGraph_t graph = nullptr;
        SG_CK(cudaGraphCreate(&graph, 0));
        long long pc = 0, pf = 0;
        const sg_status st = add_solve_loop(g, graph, S.L, S.phi, S.f, S.faces, &pc, &pf);
        if (st != SG_OK) {
            cudaGraphDestroy(graph);
            return st;
        }
        const cudaError_t ei = cudaGraphInstantiate(&g->sexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            g->sexec = nullptr;
            return fail(SG_ERR_CUDA, std::string("solve graph instantiate: ") + cudaGetErrorString(ei));
        }
        g->s_per_cycle = pc;
        g->s_per_confirm = pf;
        std::memcpy(g->skey, key, sizeof(key));
    }
    fill_device_loop(g, S, g->host_loop);
    SG_CK(cudaMemcpyAsync(g->dloop, g->host_loop, sizeof(DeviceLoop), cudaMemcpyHostToDevice, g->st));
    SG_CK(cudaGraphLaunch(g->sexec, g->st));
    SG_CK(cudaMemcpyAsync(g->host_loop, g->dloop, sizeof(DeviceLoop), cudaMemcpyDeviceToHost, g->st));
    SG_CK(cudaStreamSynchronize(g->st));
    read_device_loop(g, S, *g->host_loop, g->s_per_cycle, g->s_per_confirm);
    return SG_OK;
}

// The solve loop of sg_solve (phi, f, faces) and sg_backward (lam, w, none).
sg_status solve_impl(sg_grid* g, double tol, int L, double* phi, const double* f, bool faces,
                     bool have_guess, sg_solve_info* info) {
    SolveState S;
    SG_TRY(solve_begin(g, S, tol, L, phi, f, faces, have_guess));
    bool first = true;
    while (true) {
        SG_TRY(solve_check(g, S));
        if (S.done) break;
        if (first && use_device_loop(g, L)) {
            SG_TRY(run_device_loop(g, S));
            break;
        }
        first = false;
        bool replayed = false;
        if (L == 1) SG_TRY(solve_single_step(g, S));
        else SG_TRY(run_cycle(g, L, phi, f, faces, &replayed));
        SG_CK(cudaStreamSynchronize(g->st));
        prof_sync_point(g, replayed);
        solve_after_cycle(g, S);
    }
    return solve_end(g, S, info);
}

// With kernels (SG_HOST_COPY_KERNEL), the device address of a host buffer that
// is pinned and mapped into the device address space (cudaHostAlloc /
// cudaHostRegister memory), else nullptr (pageable memory, or copy engines
// asked for): kernels then move such buffers over the CPU-GPU link themselves,
// in one pass with any scaling, instead of a copy-engine transfer followed by
// a device pass.
const double* mapped_host(const double* p, bool kernels) {
    if (!kernels) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return static_cast<const double*>(a.devicePointer);
}

// dst (device) = scale src; src on the device or in host memory.  A host
// source may be reused by the caller once this returns.
sg_status load_scaled(double* dst, const double* src, long long n, int on_device, double scale, bool scaled,
                      cudaStream_t st, bool kernels) {
    if (on_device) {
        if (scaled) SG_CK(launch_scale_copy(src, dst, scale, n, st));
        else SG_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        return SG_OK;
    }
    if (const double* m = mapped_host(src, kernels)) {
        SG_CK(launch_link_copy(m, dst, scale, scaled, n, st));
    } else {
        SG_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, st));
        if (scaled) SG_CK(launch_scale_copy(dst, dst, scale, n, st));
    }
    SG_CK(cudaStreamSynchronize(st));
    return SG_OK;
}

sg_status copy_in(double* dst, const double* src, long long n, int on_device, cudaStream_t st, bool kernels) {
    return load_scaled(dst, src, n, on_device, 1.0, false, st, kernels);
}

sg_status copy_out(double* dst, const double* src, long long n, int on_device, cudaStream_t st, bool kernels) {
    if (on_device) {
        SG_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        return SG_OK;
    }
    if (const double* m = mapped_host(dst, kernels)) {
        SG_CK(launch_link_copy(src, const_cast<double*>(m), 1.0, false, n, st));
    } else {
        SG_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    SG_CK(cudaStreamSynchronize(st));
    return SG_OK;
}

bool kern(const sg_grid* g) { return g->opt.host_copy == SG_HOST_COPY_KERNEL; }

void free_grid(sg_grid* g) {
    if (!g) return;
    drop_graph(g);
    for (auto& L : g->lv) {
        cudaFree(L.u);
        cudaFree(L.rhs);
        cudaFree(L.z0);
        for (int i = 0; i < 3; ++i) cudaFree(L.t[i]);
    }
    cudaFree(g->phi);
    cudaFree(g->f);
    for (int i = 0; i < 6; ++i) cudaFree(g->faces[i]);
    cudaFree(g->lam);
    cudaFree(g->w);
    cudaFree(g->gphi);
    cudaFree(g->gout);
    cudaFree(g->r64);
    cudaFree(g->partials);
    cudaFree(g->red);
    cudaFree(g->d_sched);
    cudaFree(g->d_ss);
    cudaFree(g->d_mexp);
    cudaFree(g->dloop);
    if (g->host_loop) cudaFreeHost(g->host_loop);
    if (g->host_red) cudaFreeHost(g->host_red);
    if (g->host_ss) cudaFreeHost(g->host_ss);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    for (const ProfRec& r : g->live) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
    if (g->own_stream) cudaStreamDestroy(g->own_stream);
    delete g;
}

}  // namespace

// The last batch graph (sg_solve_batch): its key (serial number and graph key
// of every grid, in order), the executable graph and the kernels of one cycle
// and one confirmation per branch.
struct BatchGraph {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> per_cycle, per_confirm;
};
static BatchGraph g_batch;
static std::mutex g_batch_mu;

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

sg_status sg_default_options(sg_options* o) {
    if (!o) return fail(SG_ERR_ARG, "options pointer is NULL");
    o->rkl_order = 2;
    o->s_smooth = 3;
    o->tau_frac = 1.0;
    o->n_pre = 2;
    o->n_post = 1;
    o->coarse_tol = 1e-2;
    o->coarse_max_ss = 64;
    o->coarse_tau_frac = 0.0;
    o->max_cycles = 100;
    o->single_s = 0;
    o->single_tau_frac = 0.0;
    o->fixed_cycles = 0;
    o->use_graph = 1;
    o->fused = 1;
    o->smoother = SG_SMOOTH_RKL;
    o->omega = 1.0;
    o->max_residual_tol = 0.0;
    o->tile_rows = 0;
    o->inner_n_pre = -1;
    o->inner_n_post = -1;
    o->staging = SG_STAGE_CP_ASYNC;
    o->host_copy = SG_HOST_COPY_ENGINE;
    return SG_OK;
}

const char* sg_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {

// Grid of nx x ny x nz cells; twod: a two-dimensional grid (nz = 1, the z axis
// periodic with h_z = infinity, so 1 / h_z^2 = 0 and the z term vanishes).
sg_status create_grid(int nx, int ny, int nz, const double lo[3], const double hi[3], const int bc[3],
                      int precision, void* cuda_stream, sg_grid** out, bool twod) {
    const int n[3] = {nx, ny, nz};
    {
        // one-time kernel attributes and occupancy figures, set by whichever
        // thread creates a grid first
        static std::mutex configure_mu;
        std::lock_guard<std::mutex> lock(configure_mu);
        SG_CK(coarse_configure());
        SG_CK(fused_configure());
        SG_CK(bottom_configure());
    }
    sg_grid* g = new sg_grid();
    static std::atomic<unsigned long long> serials{0};
    g->serial = ++serials;
    g->twod = twod;
    for (int d = 0; d < 3; ++d) {
        g->n[d] = n[d];
        g->lo[d] = lo[d];
        g->hi[d] = hi[d];
        g->bc[d] = bc[d];
    }
    g->precision = precision;
    g->st = (cudaStream_t)cuda_stream;
    if (g->st == nullptr || g->st == cudaStreamLegacy) {
        // The legacy default stream cannot be captured into a CUDA graph: use a
        // private blocking stream, which the legacy stream orders implicitly.
        if (cudaStreamCreate(&g->own_stream) != cudaSuccess) {
            delete g;
            return fail(SG_ERR_CUDA, "cudaStreamCreate failed");
        }
        g->st = g->own_stream;
    }
    sg_default_options(&g->opt);
    g->max_levels = twod ? rule_levels_2d(nx, ny) : rule_levels(nx, ny, nz);
    const size_t ws = wsize(g);
    auto alloc = [&](void** p, size_t bytes) -> bool { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = true;
    long long max_blocks = kSumBlocks;
    for (int l = 0; l < g->max_levels && ok; ++l) {
        Level L;
        L.nx = nx >> l;
        L.ny = ny >> l;
        L.nz = twod ? 1 : nz >> l;
        L.n = (long long)L.nx * L.ny * L.nz;
        for (int d = 0; d < 3; ++d) L.h[d] = (hi[d] - lo[d]) / n[d] * double(1 << l);
        if (twod) L.h[2] = INFINITY;
        const bool own_u = !(l == 0 && precision == SG_FP64);
        if (own_u) ok = ok && alloc(&L.u, L.n * ws) && alloc(&L.rhs, L.n * ws);
        ok = ok && alloc(&L.z0, L.n * ws);
        for (int i = 0; i < 3; ++i) ok = ok && alloc(&L.t[i], L.n * ws);
        g->lv.push_back(L);
        const LevelGeom G = geom(g, l, false);
        max_blocks = std::max(max_blocks, residual_blocks(G));
        if (l == 0) max_blocks = std::max(max_blocks, residual_zero_blocks(geom(g, 0, true)));
        if (l + 1 < g->max_levels) max_blocks = std::max(max_blocks, restrict_blocks(G));
    }
    const long long n0 = (long long)nx * ny * nz;
    ok = ok && alloc((void**)&g->phi, n0 * sizeof(double)) && alloc((void**)&g->f, n0 * sizeof(double));
    if (precision == SG_MIXED) ok = ok && alloc((void**)&g->r64, n0 * sizeof(double));
    ok = ok && alloc((void**)&g->partials, max_blocks * sizeof(Partial));
    ok = ok && alloc((void**)&g->red, 8 * sizeof(Reduced));
    ok = ok && alloc((void**)&g->d_ss, sizeof(int));
    ok = ok && alloc((void**)&g->d_mexp, sizeof(unsigned));
    ok = ok && alloc((void**)&g->dloop, sizeof(DeviceLoop));
    ok = ok && cudaMallocHost((void**)&g->host_loop, sizeof(DeviceLoop)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&g->host_red, 8 * sizeof(Reduced)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&g->host_ss, sizeof(int)) == cudaSuccess;
    ok = ok && cudaEventCreate(&g->ev0) == cudaSuccess && cudaEventCreate(&g->ev1) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_grid(g);
        return fail(SG_ERR_OOM, "device allocation failed");
    }
    g->partial_cap = (int)max_blocks;
    const sg_status z1 = cudaMemsetAsync(g->f, 0, n0 * sizeof(double), g->st) == cudaSuccess ? SG_OK : SG_ERR_CUDA;
    const sg_status z2 = cudaMemsetAsync(g->phi, 0, n0 * sizeof(double), g->st) == cudaSuccess ? SG_OK : SG_ERR_CUDA;
    if (z1 != SG_OK || z2 != SG_OK || cudaStreamSynchronize(g->st) != cudaSuccess) {
        free_grid(g);
        return fail(SG_ERR_CUDA, "initialisation failed");
    }
    *out = g;
    return SG_OK;
}

}  // namespace

extern "C" {

sg_status sg_create_grid(int nx, int ny, int nz, const double lo[3], const double hi[3],
                         const int bc[3], int precision, void* cuda_stream, sg_grid** out) {
    g_err.clear();
    if (!out || !lo || !hi || !bc) return fail(SG_ERR_ARG, "NULL argument");
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 2 || n[d] > 4096) return fail(SG_ERR_ARG, "grid size must be in [2, 4096] per axis");
        if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
            return fail(SG_ERR_ARG, "need finite lo < hi on every axis");
        if (bc[d] != SG_BC_DIRICHLET && bc[d] != SG_BC_PERIODIC) return fail(SG_ERR_ARG, "bad boundary kind");
    }
    if ((long long)nx * ny * nz > 2147483647LL) return fail(SG_ERR_ARG, "too many cells");
    if (precision != SG_FP64 && precision != SG_MIXED) return fail(SG_ERR_ARG, "bad precision");
    return create_grid(nx, ny, nz, lo, hi, bc, precision, cuda_stream, out, false);
}

sg_status sg_create_grid_2d(int nx, int ny, const double lo[2], const double hi[2], const int bc[2], int precision,
                            void* cuda_stream, sg_grid** out) {
    g_err.clear();
    if (!out || !lo || !hi || !bc) return fail(SG_ERR_ARG, "NULL argument");
    const int n[2] = {nx, ny};
    for (int d = 0; d < 2; ++d) {
        if (n[d] < 2 || n[d] > 65536) return fail(SG_ERR_ARG, "grid size must be in [2, 65536] per axis");
        if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
            return fail(SG_ERR_ARG, "need finite lo < hi on both axes");
        if (bc[d] != SG_BC_DIRICHLET && bc[d] != SG_BC_PERIODIC) return fail(SG_ERR_ARG, "bad boundary kind");
    }
    if ((long long)nx * ny > 2147483647LL) return fail(SG_ERR_ARG, "too many cells");
    if (precision != SG_FP64 && precision != SG_MIXED) return fail(SG_ERR_ARG, "bad precision");
    const double lo3[3] = {lo[0], lo[1], 0.0}, hi3[3] = {hi[0], hi[1], 1.0};
    const int bc3[3] = {bc[0], bc[1], SG_BC_PERIODIC};
    return create_grid(nx, ny, 1, lo3, hi3, bc3, precision, cuda_stream, out, true);
}

sg_status sg_set_options(sg_grid* g, const sg_options* opt) {
    g_err.clear();
    if (!g || !opt) return fail(SG_ERR_ARG, "NULL argument");
    SG_TRY(check_opts(opt));
    g->opt = *opt;
    return SG_OK;
}

sg_status sg_get_options(const sg_grid* g, sg_options* opt) {
    if (!g || !opt) return fail(SG_ERR_ARG, "NULL argument");
    *opt = g->opt;
    return SG_OK;
}

int sg_max_levels(const sg_grid* g) { return g ? g->max_levels : 0; }

sg_status sg_plan_schedule(int N, int count, int* s_out) {
    g_err.clear();
    if (N < 1 || count < 0 || (count > 0 && !s_out)) return fail(SG_ERR_ARG, "bad schedule arguments");
    const std::vector<int> sched = accelerated_schedule(N, count);
    for (int q = 0; q < count; ++q) s_out[q] = sched[q];
    return SG_OK;
}

sg_status sg_plan_stage_coefficients(int order, int s, double* mu, double* nu, double* mut, double* gt,
                                     double* tau_max_over_dtpar) {
    g_err.clear();
    if ((order != 1 && order != 2) || s < order || s > 100000) return fail(SG_ERR_ARG, "bad order / s");
    const Rkl r = make_rkl(order, s);
    for (int j = 0; j <= s; ++j) {
        if (mu) mu[j] = r.mu[j];
        if (nu) nu[j] = r.nu[j];
        if (mut) mut[j] = r.mut[j];
        if (gt) gt[j] = r.gt[j];
    }
    if (tau_max_over_dtpar) *tau_max_over_dtpar = r.tau_over_dtpar;
    return SG_OK;
}

sg_status sg_measure_fp64_rate(double* tflops, double* ms) {
    g_err.clear();
    if (!tflops) return fail(SG_ERR_ARG, "NULL tflops");
    SG_CK(probe_fp64_rate(tflops, ms));
    return SG_OK;
}

sg_status sg_plan_s_opt(int N, int* s_out) {
    g_err.clear();
    if (N < 2 || N > 1000000 || !s_out) return fail(SG_ERR_ARG, "need 2 <= N <= 10^6 and an output pointer");
    *s_out = s_opt_global(N);
    return SG_OK;
}

int sg_plan_levels(int nx, int ny, int nz) {
    if (nx < 1 || ny < 1 || nz < 1) return 0;
    return rule_levels(nx, ny, nz);
}

sg_status sg_plan_sor_omega(int nx, int ny, int nz, const double lo[3], const double hi[3], double* omega) {
    g_err.clear();
    if (!lo || !hi || !omega || nx < 2 || ny < 2 || nz < 2) return fail(SG_ERR_ARG, "bad arguments");
    Level L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    const int n3[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        if (!(hi[d] > lo[d])) return fail(SG_ERR_ARG, "lo must be below hi on every axis");
        L.h[d] = (hi[d] - lo[d]) / n3[d];
    }
    *omega = sor_omega(L);
    return SG_OK;
}

sg_status sg_set_boundary(sg_grid* g, const double* const faces[6], int on_device) {
    g_err.clear();
    if (!g || !faces) return fail(SG_ERR_ARG, "NULL argument");
    const long long fsz[6] = {(long long)g->n[2] * g->n[1], (long long)g->n[2] * g->n[1],
                              (long long)g->n[2] * g->n[0], (long long)g->n[2] * g->n[0],
                              (long long)g->n[1] * g->n[0], (long long)g->n[1] * g->n[0]};
    for (int f = 0; f < (g->twod ? 4 : 6); ++f) {
        if (!g->faces[f]) SG_CK(cudaMalloc(&g->faces[f], fsz[f] * sizeof(double)));
        if (faces[f]) SG_TRY(copy_in(g->faces[f], faces[f], fsz[f], on_device, g->st, kern(g)));
        else SG_CK(cudaMemsetAsync(g->faces[f], 0, fsz[f] * sizeof(double), g->st));
    }
    g->have_faces = true;
    drop_graph(g);
    return SG_OK;
}

sg_status sg_set_density(sg_grid* g, const double* rho, int on_device, double four_pi_G) {
    g_err.clear();
    if (!g || !rho) return fail(SG_ERR_ARG, "NULL argument");
    if (!std::isfinite(four_pi_G)) return fail(SG_ERR_ARG, "four_pi_G must be finite");
    const long long n = g->lv[0].n;
    SG_TRY(load_scaled(g->f, rho, n, on_device, four_pi_G, true, g->st, kern(g)));
    if (all_periodic(g)) {                      // Eq. source_modification
        int nb = 0;
        SG_CK(launch_sum_partials_f64(g->f, n, g->partials, &nb, g->st));
        SG_CK(launch_finalize(g->partials, nb, g->red + 1, g->st));
        SG_CK(launch_sub_mean_f64(g->f, n, g->red + 1, g->st));
    }
    g->four_pi_G = four_pi_G;
    g->have_density = true;
    g->guess_set = false;
    return SG_OK;
}

sg_status sg_set_potential_guess(sg_grid* g, const double* phi, int on_device) {
    g_err.clear();
    if (!g || !phi) return fail(SG_ERR_ARG, "NULL argument");
    SG_TRY(copy_in(g->phi, phi, g->lv[0].n, on_device, g->st, kern(g)));
    g->guess_set = true;
    return SG_OK;
}

sg_status sg_solve(sg_grid* g, double tol, int s, int levels, sg_solve_info* info) {
    g_err.clear();
    if (!g) return fail(SG_ERR_ARG, "NULL grid");
    if (!(tol >= 0.0)) return fail(SG_ERR_ARG, "tol must be >= 0");
    if (levels < 0 || levels > g->max_levels) return fail(SG_ERR_ARG, "levels exceeds the level rule");
    if (s < 0) return fail(SG_ERR_ARG, "s must be >= 0");
    if (!g->have_density) return fail(SG_ERR_STATE, "sg_set_density first");
    const int L = levels == 0 ? g->max_levels : levels;
    sg_options saved = g->opt;
    if (s > 0) {
        if (L == 1) g->opt.single_s = s;
        else g->opt.s_smooth = s;
        const sg_status c = check_opts(&g->opt);
        if (c != SG_OK) {
            g->opt = saved;
            return c;
        }
    }
    const bool faces = g->have_faces;
    const sg_status st = solve_impl(g, tol, L, g->phi, g->f, faces, g->guess_set, info);
    g->opt = saved;
    g->guess_set = false;
    if (st == SG_OK || st == SG_ERR_NOT_CONVERGED) {
        g->have_solution = true;
        g->last_levels = L;
    }
    return st;
}

sg_status sg_gravity(sg_grid* g, const double* phi, double* g_out, int on_device) {
    g_err.clear();
    if (!g || !g_out) return fail(SG_ERR_ARG, "NULL argument");
    if (!phi && !g->have_solution) return fail(SG_ERR_STATE, "no solution yet");
    const long long n = g->lv[0].n;
    if (phi && on_device) {
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(phi), b0 = reinterpret_cast<uintptr_t>(g_out);
        if (a0 < b0 + 3 * n * sizeof(double) && b0 < a0 + n * sizeof(double))
            return fail(SG_ERR_ARG, "g_out overlaps phi");
    }
    const double* src = phi ? phi : g->phi;
    if (phi && !on_device) {
        if (!g->gphi) SG_CK(cudaMalloc(&g->gphi, n * sizeof(double)));
        SG_TRY(copy_in(g->gphi, phi, n, 0, g->st, kern(g)));
        src = g->gphi;
    }
    double* dst = g_out;
    if (!on_device) {
        if (!g->gout) SG_CK(cudaMalloc(&g->gout, 3 * n * sizeof(double)));
        dst = g->gout;
    }
    const Level& L0 = g->lv[0];
    const double c[3] = {-1.0 / (12.0 * L0.h[0]), -1.0 / (12.0 * L0.h[1]), -1.0 / (12.0 * L0.h[2])};
    int nk = 1;
    {
        ProfScope ps(g, K_GRAVITY, 32.0 * n);
        SG_CK(launch_gravity(geom(g, 0, g->have_faces), src, dst, c, g->d_mexp, &nk, g->st));
    }
    g->launches += nk;
    if (!on_device) SG_TRY(copy_out(g_out, dst, 3 * n, 0, g->st, kern(g)));
    return SG_OK;
}

sg_status sg_potential(sg_grid* g, double* phi_out, int on_device) {
    g_err.clear();
    if (!g || !phi_out) return fail(SG_ERR_ARG, "NULL argument");
    if (!g->have_solution) return fail(SG_ERR_STATE, "no solution yet");
    return copy_out(phi_out, g->phi, g->lv[0].n, on_device, g->st, kern(g));
}

sg_status sg_backward(sg_grid* g, const double* dL_dphi, double* dL_drho, int on_device, double tol,
                      sg_solve_info* info) {
    g_err.clear();
    if (!g || !dL_dphi || !dL_drho) return fail(SG_ERR_ARG, "NULL argument");
    if (!(tol >= 0.0)) return fail(SG_ERR_ARG, "tol must be >= 0");
    const long long n = g->lv[0].n;
    if (!g->lam) SG_CK(cudaMalloc(&g->lam, n * sizeof(double)));
    if (!g->w) SG_CK(cudaMalloc(&g->w, n * sizeof(double)));
    SG_TRY(copy_in(g->w, dL_dphi, n, on_device, g->st, kern(g)));
    if (all_periodic(g)) {
        int nb = 0;
        SG_CK(launch_sum_partials_f64(g->w, n, g->partials, &nb, g->st));
        SG_CK(launch_finalize(g->partials, nb, g->red + 1, g->st));
        SG_CK(launch_sub_mean_f64(g->w, n, g->red + 1, g->st));
    }
    const int L = g->last_levels > 0 ? g->last_levels : g->max_levels;
    const sg_status st = solve_impl(g, tol, L, g->lam, g->w, false, false, info);
    if (st != SG_OK && st != SG_ERR_NOT_CONVERGED) return st;
    SG_CK(launch_scale_copy(g->lam, g->lam, g->four_pi_G, n, g->st));
    SG_TRY(copy_out(dL_drho, g->lam, n, on_device, g->st, kern(g)));
    return st;
}

sg_status sg_solve_batch(sg_grid* const* grids, int n, double tol, sg_solve_info* infos) {
    g_err.clear();
    if (!grids || n < 0) return fail(SG_ERR_ARG, "bad batch arguments");
    if (!(tol >= 0.0)) return fail(SG_ERR_ARG, "tol must be >= 0");
    for (int i = 0; i < n; ++i) {
        if (!grids[i]) return fail(SG_ERR_ARG, "NULL grid in batch");
        if (!grids[i]->have_density) return fail(SG_ERR_STATE, "sg_set_density first (batch)");
        for (int k = 0; k < i; ++k)
            if (grids[k] == grids[i]) return fail(SG_ERR_ARG, "a grid appears twice in the batch");
    }
    sg_status first = SG_OK;
    // Grids whose cycle loop can run on the device become one branch each of a
    // single graph (sg_solve's loop: WHILE nodes decided on the device); the
    // rest (single level, coarsest level too large for one CTA, graph replay
    // disabled, profiling on) are solved one after the other.
    std::vector<int> par;
    for (int i = 0; i < n; ++i) {
        sg_grid* g = grids[i];
        if (use_device_loop(g, g->max_levels)) {
            par.push_back(i);
        } else {
            const sg_status st = sg_solve(g, tol, 0, 0, infos ? &infos[i] : nullptr);
            if (st != SG_OK && first == SG_OK) first = st;
        }
    }
    if (par.empty()) return first;
    const size_t P = par.size();
    std::vector<SolveState> S(P);
    for (size_t k = 0; k < P; ++k) {
        sg_grid* g = grids[par[k]];
        SG_TRY(solve_begin(g, S[k], tol, g->max_levels, g->phi, g->f, g->have_faces, g->guess_set));
        g->guess_set = false;
        SG_TRY(solve_check(g, S[k]));
    }
    // the batch graph, kept while the same grids (by serial number) with the
    // same keys come back
    std::vector<uint64_t> key;
    for (size_t k = 0; k < P; ++k) {
        sg_grid* g = grids[par[k]];
        uint64_t gk[kGraphKeySlots];
        graph_key(g, S[k].L, S[k].phi, S[k].f, S[k].faces, gk);
        key.push_back(g->serial);
        key.insert(key.end(), gk, gk + kGraphKeySlots);
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    cudaStream_t origin = grids[par[0]]->st;
    if (!g_batch.exec || g_batch.key != key) {
        if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
        g_batch.exec = nullptr;
        g_batch.key.clear();
        cudaGraph_t graph = nullptr;
        SG_CK(cudaGraphCreate(&graph, 0));
        g_batch.per_cycle.assign(P, 0);
        g_batch.per_confirm.assign(P, 0);
        for (size_t k = 0; k < P; ++k) {
            sg_grid* g = grids[par[k]];
            const sg_status st = add_solve_loop(g, graph, S[k].L, S[k].phi, S[k].f, S[k].faces,
                                                &g_batch.per_cycle[k], &g_batch.per_confirm[k]);
            if (st != SG_OK) {
                cudaGraphDestroy(graph);
                return st;
            }
        }
        const cudaError_t ei = cudaGraphInstantiate(&g_batch.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            g_batch.exec = nullptr;
            return fail(SG_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(ei));
        }
        g_batch.key = key;
    }
    for (size_t k = 0; k < P; ++k) {
        sg_grid* g = grids[par[k]];
        fill_device_loop(g, S[k], g->host_loop);
        SG_CK(cudaMemcpyAsync(g->dloop, g->host_loop, sizeof(DeviceLoop), cudaMemcpyHostToDevice, origin));
    }
    SG_CK(cudaGraphLaunch(g_batch.exec, origin));
    for (size_t k = 0; k < P; ++k) {
        sg_grid* g = grids[par[k]];
        SG_CK(cudaMemcpyAsync(g->host_loop, g->dloop, sizeof(DeviceLoop), cudaMemcpyDeviceToHost, origin));
    }
    SG_CK(cudaStreamSynchronize(origin));
    for (size_t k = 0; k < P; ++k) {
        sg_grid* g = grids[par[k]];
        read_device_loop(g, S[k], *g->host_loop, g_batch.per_cycle[k], g_batch.per_confirm[k]);
        const sg_status st = solve_end(g, S[k], infos ? &infos[par[k]] : nullptr);
        if (st == SG_OK || st == SG_ERR_NOT_CONVERGED) {
            g->have_solution = true;
            g->last_levels = S[k].L;
        }
        if (st != SG_OK && first == SG_OK) first = st;
    }
    return first;
}

sg_status sg_autotune(sg_grid* g, int levels, int keep_order, sg_tune_entry* table, int cap, int* count) {
    g_err.clear();
    if (!g) return fail(SG_ERR_ARG, "NULL grid");
    if (!g->have_density) return fail(SG_ERR_STATE, "sg_set_density first");
    if (levels < 0 || levels > g->max_levels) return fail(SG_ERR_ARG, "levels exceeds the level rule");
    const int L = levels == 0 ? g->max_levels : levels;
    if (L < 2) return fail(SG_ERR_ARG, "autotuning needs a multigrid hierarchy (levels >= 2)");
    const sg_options saved = g->opt;
    struct Cand { int order, s, fused; double c; int pre, post, rows, ipre, ipost; };
    std::vector<Cand> cands;
    // more smoothing per cycle trades the cycle's fixed work (update,
    // transfers, coarsest levels) against fewer cycles
    const int counts[][2] = {{2, 1}, {3, 2}, {4, 3}, {5, 3}};
    for (int order = 1; order <= 2; ++order) {
        if (keep_order && order != saved.rkl_order) continue;
        for (int s = 2; s <= 6; ++s) {
            const double cs1[] = {0.6, 0.75, 0.9};
            const double cs2[] = {0.8, 0.9, 1.0};
            const double* cs = order == 1 ? cs1 : cs2;
            for (int ic = 0; ic < 3; ++ic)
                for (int fz = 0; fz <= (g->precision == SG_MIXED ? 1 : 0); ++fz)
                    for (const auto& pc : counts)
                        for (int in = 0; in < 2; ++in) {      // inner levels: the same counts, or (2, 1)
                            const int ip = in ? 2 : -1, iq = in ? 1 : -1;
                            if (in && pc[0] == 2 && pc[1] == 1) continue;
                            if (fz && s <= 3 && !g->twod) {      // the tile shapes of the fused s = 2, 3 kernel
                                cands.push_back({order, s, fz, cs[ic], pc[0], pc[1], 14, ip, iq});
                                cands.push_back({order, s, fz, cs[ic], pc[0], pc[1], 16, ip, iq});
                            } else {
                                cands.push_back({order, s, fz, cs[ic], pc[0], pc[1], 0, ip, iq});
                            }
                        }
        }
    }
    double best = 1e300;
    sg_options best_opt = saved;
    int tried = 0;
    for (const Cand& c : cands) {
        g->opt = saved;
        g->opt.rkl_order = c.order;
        g->opt.s_smooth = c.s;
        g->opt.tau_frac = c.c;
        g->opt.fused = c.fused;
        g->opt.n_pre = c.pre;
        g->opt.n_post = c.post;
        g->opt.tile_rows = c.rows;
        g->opt.inner_n_pre = c.ipre;
        g->opt.inner_n_post = c.ipost;
        g->opt.smoother = SG_SMOOTH_RKL;
        // Time 2 and 6 cycles (after a capture / warm-up run) and take the
        // difference, so the per-solve set-up cost drops out of the score.
        sg_solve_info info2, info6;
        sg_status st = SG_OK;
        for (int rep = 0; rep < 3 && st == SG_OK; ++rep) {
            g->opt.fixed_cycles = rep == 2 ? 6 : 2;
            st = solve_impl(g, 0.0, L, g->phi, g->f, g->have_faces, false, rep == 2 ? &info6 : &info2);
        }
        if (st != SG_OK) {
            g->opt = saved;
            return st;
        }
        const double h2 = info6.history[2], h6 = info6.history[6];
        double factor = (h2 > 0 && h6 > 0) ? std::pow(h6 / h2, 0.25) : 1.0;
        // The checkerboard mode restricts to zero, so only the smoother acts on
        // it: its factor per cycle bounds the asymptotic rate from below (RKL2
        // with even s at tau_max leaves it untouched, which a few early cycles
        // do not show).
        const double top = std::pow(std::fabs(rkl_top_amplification(make_rkl(c.order, c.s), c.c)),
                                    double(g->opt.n_pre + g->opt.n_post));
        factor = std::max(factor, top);
        const double mpc = (info6.elapsed_ms - info2.elapsed_ms) / 4.0;
        const double score = (factor > 0 && factor < 1) ? mpc / -std::log10(factor) : 1e300;
        if (table && tried < cap)
            table[tried] = {c.order, c.s, c.fused, c.c, mpc, factor, score, c.pre, c.post, c.rows, c.ipre, c.ipost};
        (void)info2;
        ++tried;
        if (score < best) {
            best = score;
            best_opt = g->opt;
        }
    }
    best_opt.fixed_cycles = saved.fixed_cycles;
    g->opt = best_opt;
    g->have_solution = false;
    if (count) *count = tried;
    return SG_OK;
}

void sg_destroy(sg_grid* g) { free_grid(g); }

sg_status sg_set_profiling(sg_grid* g, int on) {
    g_err.clear();
    if (!g) return fail(SG_ERR_ARG, "NULL grid");
    g->prof = on != 0;
    drop_graph(g);
    for (int c = 0; c < K_NCLASS; ++c) {
        std::memset(&g->stats[c], 0, sizeof(sg_kernel_stat));
        std::snprintf(g->stats[c].name, sizeof(g->stats[c].name), "%s", kClassName[c]);
    }
    return SG_OK;
}

sg_status sg_kernel_stats(sg_grid* g, sg_kernel_stat* out) {
    g_err.clear();
    if (!g || !out) return fail(SG_ERR_ARG, "NULL argument");
    if (g->prof && !g->live.empty() && !g->capturing) {
        // launches recorded since the last solve's sync point (single operators, sg_gravity)
        SG_CK(cudaStreamSynchronize(g->st));
        prof_accumulate(g, g->live, true);
    }
    for (int c = 0; c < K_NCLASS; ++c) {
        out[c] = g->stats[c];
        std::snprintf(out[c].name, sizeof(out[c].name), "%s", kClassName[c]);
    }
    return SG_OK;
}

// ---- single operators --------------------------------------------------------
static sg_status op_check(sg_grid* g, int level, int dtype) {
    if (!g) return fail(SG_ERR_ARG, "NULL grid");
    if (level < 0 || level >= g->max_levels) return fail(SG_ERR_ARG, "level out of range");
    if (dtype != 0 && dtype != 1) return fail(SG_ERR_ARG, "dtype must be 0 (f64) or 1 (f32)");
    const bool w64 = g->precision == SG_FP64;
    if ((dtype == 0) != w64) return fail(SG_ERR_ARG, "dtype must match the grid's working precision");
    return SG_OK;
}

sg_status sg_op_superstep(sg_grid* g, int level, int dtype, int order, int s, double tau_frac,
                          int homogeneous, const void* u, const void* rhs, void* out) {
    g_err.clear();
    SG_TRY(op_check(g, level, dtype));
    if (!rhs || !out || out == u || out == rhs) return fail(SG_ERR_ARG, "bad pointers");
    if ((order != 1 && order != 2) || s < 1 || (order == 2 && s < 2) || !(tau_frac > 0 && tau_frac <= 1))
        return fail(SG_ERR_ARG, "bad order / s / tau_frac");
    const bool faces = !homogeneous && level == 0 && g->have_faces;
    if (dtype == 1 && g->opt.fused && !faces && !g->twod && fused_supported(order, s))
        return superstep_fused(g, level, order, s, tau_frac, (const float*)u, (const float*)rhs, (float*)out);
    if (!u) return fail(SG_ERR_ARG, "u == NULL (zero initial guess) needs the fused FP32 super-step");
    const size_t bytes = g->lv[level].n * (dtype == 0 ? 8 : 4);
    SG_CK(cudaMemcpyAsync(out, u, bytes, cudaMemcpyDeviceToDevice, g->st));
    if (dtype == 0) return superstep<double>(g, level, order, s, tau_frac, faces, (double*)out, (const double*)rhs);
    return superstep<float>(g, level, order, s, tau_frac, faces, (float*)out, (const float*)rhs);
}

sg_status sg_op_gsrb_sweep(sg_grid* g, int level, int dtype, int homogeneous, double omega, void* u,
                           const void* rhs) {
    g_err.clear();
    SG_TRY(op_check(g, level, dtype));
    if (!u || !rhs || u == rhs) return fail(SG_ERR_ARG, "bad pointers");
    if (!(omega >= 0.0 && omega < 2.0)) return fail(SG_ERR_ARG, "omega must be in [0, 2)");
    const Level& Lv = g->lv[level];
    const int n3[3] = {Lv.nx, Lv.ny, Lv.nz};
    for (int d = 0; d < 3; ++d)
        if (g->bc[d] == SG_BC_PERIODIC && (n3[d] & 1))
            return fail(SG_ERR_ARG, "GS-RB needs even extents on periodic axes");
    const bool faces = !homogeneous && level == 0 && g->have_faces;
    const double om = omega > 0.0 ? omega : sor_omega(Lv);
    if (dtype == 0) return gsrb_sweep<double>(g, level, faces, (double*)u, (const double*)rhs, om);
    return gsrb_sweep<float>(g, level, faces, (float*)u, (const float*)rhs, om);
}

sg_status sg_op_residual_restrict(sg_grid* g, int level, int dtype, int homogeneous, const void* u,
                                  const void* rhs, void* coarse_out, double norms[2]) {
    g_err.clear();
    SG_TRY(op_check(g, level, dtype));
    if (!u || !rhs) return fail(SG_ERR_ARG, "bad pointers");
    if (coarse_out && level + 1 >= g->max_levels) return fail(SG_ERR_ARG, "no coarser level");
    const bool faces = !homogeneous && level == 0 && g->have_faces;
    const LevelGeom G = geom(g, level, faces);
    int nb = 0;
    if (coarse_out) {
        if (dtype == 0)
            SG_CK(launch_residual_restrict<double>(G, (const double*)u, (const double*)rhs, (double*)coarse_out,
                                                   g->partials, &nb, g->st));
        else
            SG_CK(launch_residual_restrict<float>(G, (const float*)u, (const float*)rhs, (float*)coarse_out,
                                                  g->partials, &nb, g->st));
    } else {
        if (dtype == 0)
            SG_CK(launch_residual<double, double>(G, (const double*)u, (const double*)rhs, (double*)nullptr,
                                                  g->partials, &nb, g->st));
        else
            SG_CK(launch_residual<float, float>(G, (const float*)u, (const float*)rhs, (float*)nullptr,
                                                g->partials, &nb, g->st));
    }
    if (norms) {
        SG_CK(launch_finalize(g->partials, nb, g->red + 4, g->st));
        SG_CK(cudaMemcpyAsync(g->host_red + 4, g->red + 4, sizeof(Reduced), cudaMemcpyDeviceToHost, g->st));
        SG_CK(cudaStreamSynchronize(g->st));
        norms[0] = g->host_red[4].sumsq;
        norms[1] = g->host_red[4].maxabs;
    }
    return SG_OK;
}

sg_status sg_op_residual_exact(sg_grid* g, int homogeneous, const double* u, const double* rhs, double* r_out,
                               float* r32_out, double norms[2]) {
    g_err.clear();
    if (!g) return fail(SG_ERR_ARG, "null grid");
    if (!u || !rhs || !r_out || !r32_out) return fail(SG_ERR_ARG, "bad pointers");
    const bool faces = !homogeneous && g->have_faces;
    const LevelGeom G = geom(g, 0, faces);
    int nb = 0, nk = 1;
    SG_CK(launch_residual_exact(G, u, rhs, r32_out, r_out, g->partials, g->d_mexp, &nb, &nk, g->st));
    g->launches += nk;
    if (norms) {
        SG_CK(launch_finalize(g->partials, nb, g->red + 4, g->st));
        SG_CK(cudaMemcpyAsync(g->host_red + 4, g->red + 4, sizeof(Reduced), cudaMemcpyDeviceToHost, g->st));
        SG_CK(cudaStreamSynchronize(g->st));
        norms[0] = g->host_red[4].sumsq;
        norms[1] = g->host_red[4].maxabs;
    }
    return SG_OK;
}

sg_status sg_op_prolong_correct(sg_grid* g, int level, int dtype, const void* coarse, void* fine) {
    g_err.clear();
    SG_TRY(op_check(g, level, dtype));
    if (!coarse || !fine) return fail(SG_ERR_ARG, "bad pointers");
    if (level + 1 >= g->max_levels) return fail(SG_ERR_ARG, "no coarser level");
    const LevelGeom G = geom(g, level, false);
    if (dtype == 0) SG_CK(launch_prolong_correct<double>(G, (const double*)coarse, (double*)fine, g->st));
    else SG_CK(launch_prolong_correct<float>(G, (const float*)coarse, (float*)fine, g->st));
    return SG_OK;
}

sg_status sg_op_coarse_solve(sg_grid* g, int level, int dtype, const void* rhs, void* u_out, int* ss_done) {
    g_err.clear();
    SG_TRY(op_check(g, level, dtype));
    if (!rhs || !u_out) return fail(SG_ERR_ARG, "bad pointers");
    const Level& L = g->lv[level];
    const int N = std::max(L.nx, std::max(L.ny, L.nz));
    SG_TRY(ensure_sched(g, accelerated_schedule(N, g->opt.coarse_max_ss)));
    if (dtype == 0) SG_TRY(coarse_solve<double>(g, level, (const double*)rhs, (double*)u_out, g->d_ss));
    else SG_TRY(coarse_solve<float>(g, level, (const float*)rhs, (float*)u_out, g->d_ss));
    if (ss_done) {
        SG_CK(cudaMemcpyAsync(g->host_ss, g->d_ss, sizeof(int), cudaMemcpyDeviceToHost, g->st));
        SG_CK(cudaStreamSynchronize(g->st));
        *ss_done = *g->host_ss;
    }
    return SG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free residual, restriction and norms (sg_residual_restrict_noalloc).
//
// Some callers may not allocate device memory while they run: a job whose
// memory is reserved up front (a caching allocator holding the whole device, a
// real-time loop), or a host that owns only its arrays and wants no grid object
// (creating one allocates every multigrid level).  This entry point runs the
// same residual / residual-restrict and norm-fold kernels as
// sg_op_residual_restrict, but the per-block partial norms and the folded
// result live in one array compiled into this library, so it calls no
// allocating routine.
// ---------------------------------------------------------------------------
namespace {

constexpr int kStaticSlots = 8192;                                 // per-block partial norms
constexpr size_t kStaticRedOffset = size_t(kStaticSlots) * sizeof(Partial);
constexpr size_t kStaticBytes = kStaticRedOffset + 256;            // + the folded Reduced
static_assert(kStaticRedOffset % 256 == 0 && sizeof(Reduced) <= 256, "static scratch layout");
constexpr int kStaticMaxDevices = 64;

}  // namespace

// 256 KiB + 256 B per device, shared by every call on that device.
static __device__ __align__(256) unsigned char sg_static_scratch[kStaticBytes];

namespace {

std::mutex g_static_mu;
unsigned char* g_static_addr[kStaticMaxDevices] = {};

// Device address of the scratch on the current device; looked up once per
// device (the lookup may load this library's kernels onto that device).
sg_status static_scratch(unsigned char** out) {
    int dev = -1;
    SG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStaticMaxDevices) return fail(SG_ERR_ARG, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, sg_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(SG_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        g_static_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_addr[dev];
    return SG_OK;
}

}  // namespace

extern "C" sg_status sg_residual_restrict_noalloc(int nx, int ny, int nz, const double lo[3], const double hi[3],
                                                  const int bc[3], const double* const faces[6], int dtype,
                                                  const void* u, const void* rhs, void* coarse_out, double norms[2],
                                                  void* cuda_stream) {
    g_err.clear();
    if (!lo || !hi || !bc) return fail(SG_ERR_ARG, "NULL lo, hi or bc");
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 2 || n[d] > 4096) return fail(SG_ERR_ARG, "grid size must be in [2, 4096] per axis");
        if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
            return fail(SG_ERR_ARG, "need finite lo < hi on every axis");
        if (bc[d] != SG_BC_DIRICHLET && bc[d] != SG_BC_PERIODIC) return fail(SG_ERR_ARG, "bad boundary kind");
    }
    if ((long long)nx * ny * nz > 2147483647LL) return fail(SG_ERR_ARG, "too many cells");
    if (dtype != 0 && dtype != 1) return fail(SG_ERR_ARG, "dtype must be 0 (float64) or 1 (float32)");
    if (!u || !rhs) return fail(SG_ERR_ARG, "bad pointers");
    if (!coarse_out && !norms) return fail(SG_ERR_ARG, "nothing to compute: coarse_out and norms are both NULL");
    if (coarse_out && ((nx | ny | nz) & 1)) return fail(SG_ERR_ARG, "restriction needs even sizes on every axis");

    LevelGeom G;
    G.nx = nx;
    G.ny = ny;
    G.nz = nz;
    double ih2[3];
    for (int d = 0; d < 3; ++d) {
        const double h = (hi[d] - lo[d]) / n[d];
        ih2[d] = 1.0 / (h * h);
        G.per[d] = bc[d] == SG_BC_PERIODIC;
    }
    G.ihx2 = ih2[0];
    G.ihy2 = ih2[1];
    G.ihz2 = ih2[2];
    G.ihx2f = float(G.ihx2);
    G.ihy2f = float(G.ihy2);
    G.ihz2f = float(G.ihz2);
    for (int f = 0; f < 6; ++f) G.face[f] = (faces && bc[f / 2] == SG_BC_DIRICHLET) ? faces[f] : nullptr;
    G.twod = 0;

    const long long need = coarse_out ? restrict_blocks(G) : residual_blocks(G);
    if (need > kStaticSlots)
        return fail(SG_ERR_ARG, "this grid needs " + std::to_string(need) + " block slots; the static scratch holds " +
                                    std::to_string(kStaticSlots));

    unsigned char* base = nullptr;
    SG_TRY(static_scratch(&base));
    Partial* partials = reinterpret_cast<Partial*>(base);
    Reduced* red = reinterpret_cast<Reduced*>(base + kStaticRedOffset);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // Every launched block writes its own slot before the fold reads it, and
    // the fold writes the whole result: nothing here needs clearing.
    int nb = 0;
    if (coarse_out) {
        if (dtype == 0)
            SG_CK(launch_residual_restrict<double>(G, (const double*)u, (const double*)rhs, (double*)coarse_out,
                                                   partials, &nb, st));
        else
            SG_CK(launch_residual_restrict<float>(G, (const float*)u, (const float*)rhs, (float*)coarse_out,
                                                  partials, &nb, st));
    } else {
        if (dtype == 0)
            SG_CK(launch_residual<double, double>(G, (const double*)u, (const double*)rhs, (double*)nullptr,
                                                  partials, &nb, st));
        else
            SG_CK(launch_residual<float, float>(G, (const float*)u, (const float*)rhs, (float*)nullptr,
                                                partials, &nb, st));
    }
    if (norms) {
        SG_CK(launch_finalize(partials, nb, red, st));
        Reduced h{};
        SG_CK(cudaMemcpyAsync(&h, red, sizeof(Reduced), cudaMemcpyDeviceToHost, st));
        SG_CK(cudaStreamSynchronize(st));
        norms[0] = h.sumsq;
        norms[1] = h.maxabs;
    }
    return SG_OK;
}
