// The two coarsest levels of the FP32 V-cycle in one launch (Sec. 2.1 steps
// 2c-2e and 3, Eq. RKL_intermediate_source, App. A.5): a thread-block cluster
// holds level B (the second coarsest) and level C = B + 1 (the coarsest) in
// distributed shared memory and runs, without touching global memory between
// them,
//   the n_pre smoothing super-steps of B from e_B = 0,
//   r_B = f_B - L e_B and its 8-child restriction f_C (mean removed when every
//   axis is periodic, Eq. source_modification),
//   the accelerated RKL1 solve of L e_C = f_C from e_C = 0 (schedule s_k,
//   stopped by the coarse tolerance),
//   e_B += P e_C (27/9/3/1 prolongation) and the n_post smoothing super-steps.
//
// Layout.  CTA `rank` of the cluster owns the z slab [rank pz, (rank + 1) pz)
// of level B and the matching slab of pz / 2 planes of level C; every field is
// stored with a one-cell ghost layer.  A thread owns one (x, y) column of the
// slab.  Ghosts follow the boundary rule of the level (Eq. error_ghost: ghost =
// -active; Eq. periodic: the opposite cell): the thread writing a boundary cell
// writes the x / y ghost in its own CTA and the z ghost plane of the
// neighbouring CTA (through distributed shared memory), and a cluster barrier
// (release / acquire) ends every stage.  Block and cluster sums are folded in
// a fixed order and every CTA folds the same partials, so all CTAs take the
// same stop decision and pass the same barriers.
//
// The arithmetic of every stage, of the residual, the restriction and the
// prolongation is written in the order of the single-level kernels.
#include "sg_internal.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace sg {

namespace {

constexpr int kBottomMaxNC = 8;          // CTAs per cluster (portable size)
constexpr size_t kSmemLimit = 227u * 1024u - 1024u;   // dynamic shared memory per CTA

__device__ __forceinline__ float lap7f(float c, float xm, float xp, float ym, float yp, float zm, float zp, float hx,
                                       float hy, float hz) {
    const float two_c = 2.0f * c;
    return ((xm - two_c) + xp) * hx + ((ym - two_c) + yp) * hy + ((zm - two_c) + zp) * hz;
}

// A field of one level: (pz + 2) planes of (ny + 2) rows of (nx + 2) floats.
struct Slab {
    int nx, ny, pz, row, plane;
    __device__ int at(int k, int j, int i) const { return (k + 1) * plane + (j + 1) * row + (i + 1); }
};

__device__ __forceinline__ Slab make_slab(int nx, int ny, int pz) {
    Slab s;
    s.nx = nx;
    s.ny = ny;
    s.pz = pz;
    s.row = nx + 2;
    s.plane = (nx + 2) * (ny + 2);
    return s;
}

struct Ctx {
    cg::cluster_group cl;
    int rank, nc;
    bool px, py, pz;
};

// v at interior cell (k, j, i) of field `f` (offset in the CTA's shared
// memory), with the x / y ghosts of this CTA and the z ghost plane of the
// neighbouring CTA (or of this CTA at a wall).
__device__ __forceinline__ void put(const Ctx& c, float* sm, int f, const Slab& s, int k, int j, int i, float v) {
    float* fl = sm + f;
    fl[s.at(k, j, i)] = v;
    if (i == 0) fl[s.at(k, j, c.px ? s.nx : -1)] = c.px ? v : -v;
    if (i == s.nx - 1) fl[s.at(k, j, c.px ? -1 : s.nx)] = c.px ? v : -v;
    if (j == 0) fl[s.at(k, c.py ? s.ny : -1, i)] = c.py ? v : -v;
    if (j == s.ny - 1) fl[s.at(k, c.py ? -1 : s.ny, i)] = c.py ? v : -v;
    if (k == 0) {
        if (c.rank > 0 || c.pz) {
            const int peer = c.rank > 0 ? c.rank - 1 : c.nc - 1;
            float* r = c.cl.map_shared_rank(sm, peer) + f;
            r[s.at(s.pz, j, i)] = v;
        } else {
            fl[s.at(-1, j, i)] = -v;
        }
    }
    if (k == s.pz - 1) {
        if (c.rank < c.nc - 1 || c.pz) {
            const int peer = c.rank < c.nc - 1 ? c.rank + 1 : 0;
            float* r = c.cl.map_shared_rank(sm, peer) + f;
            r[s.at(-1, j, i)] = v;
        } else {
            fl[s.at(s.pz, j, i)] = -v;
        }
    }
}

__device__ __forceinline__ float lap_at(const float* y, const Slab& s, int k, int j, int i, float hx, float hy,
                                        float hz) {
    const int o = s.at(k, j, i);
    return lap7f(y[o], y[o - 1], y[o + 1], y[o - s.row], y[o + s.row], y[o - s.plane], y[o + s.plane], hx, hy, hz);
}

// Sum of v over the block, fixed order; every thread gets the result.
__device__ __forceinline__ float block_sum(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();                             // red is free (previous readers done)
    if (lane == 0) red[w] = v;
    __syncthreads();
    float t = 0.0f;
    for (int k = 0; k < nw; ++k) t += red[k];
    return t;
}

// Sum over the cluster: every CTA's block sum, folded in rank order by every
// CTA.  Partials alternate between two slot arrays, so a CTA writing the next
// round never overwrites slots a peer is still reading.
__device__ __forceinline__ float cluster_sum(const Ctx& c, float* sm, int cred, int& round, float v, float* red) {
    const float b = block_sum(v, red);
    const int slot = cred + (round & 1) * kBottomMaxNC;
    if (threadIdx.x < c.nc) {
        float* r = c.cl.map_shared_rank(sm, (int)threadIdx.x) + slot;
        r[c.rank] = b;
    }
    ++round;
    c.cl.sync();
    float t = 0.0f;
    for (int k = 0; k < c.nc; ++k) t += sm[slot + k];
    return t;
}

__global__ void __launch_bounds__(1024) k_bottom_levels(const __grid_constant__ BottomParams p) {
    extern __shared__ __align__(16) float sm[];
    __shared__ float red[32];
    Ctx c{cg::this_cluster(), 0, 0, p.per[0] != 0, p.per[1] != 0, p.per[2] != 0};
    c.rank = (int)c.cl.block_rank();
    c.nc = (int)c.cl.num_blocks();
    const int nx = p.nx, ny = p.ny, nz = p.nz, pz = nz / c.nc;
    const int cnx = nx / 2, cny = ny / 2, cpz = pz / 2;
    const Slab sb = make_slab(nx, ny, pz), sc = make_slab(cnx, cny, cpz);
    const int fb = sb.plane * (pz + 2), fc = sc.plane * (cpz + 2);
    // fields: level B rhs, Z0 / residual, four iterates; level C rhs, three iterates; cluster partials
    const int F = 0, Z = fb, YB = 2 * fb;
    const int FC = 6 * fb, YC = FC + fc, CRED = FC + 4 * fc;
    const int nfl = CRED + 2 * kBottomMaxNC;
    const int tid = threadIdx.x;
    const bool act_b = tid < nx * ny, act_c = tid < cnx * cny;
    const int i = act_b ? tid % nx : 0, j = act_b ? tid / nx : 0;
    const int I = act_c ? tid % cnx : 0, J = act_c ? tid / cnx : 0;
    const float hx = p.hx, hy = p.hy, hz = p.hz;
    int round = 0;

    for (int t = tid; t < nfl; t += blockDim.x) sm[t] = 0.0f;
    c.cl.sync();                                 // no peer writes a ghost before it is cleared
    if (act_b)
        for (int k = 0; k < pz; ++k) sm[F + sb.at(k, j, i)] = p.rhs[((size_t)(c.rank * pz + k) * ny + j) * nx + i];
    __syncthreads();

    // ---- smoothing super-steps of level B (App. A, Eq. RKL_intermediate_source)
    int e = YB;                                   // current iterate (zero)
    int spare[3] = {YB + fb, YB + 2 * fb, YB + 3 * fb};
    auto superstep = [&]() {
        const int y0 = e;
        for (int js = 1; js <= p.s; ++js) {
            const int out = spare[(js - 1) % 3];
            const int ym1 = js == 1 ? y0 : spare[(js - 2) % 3];
            const int ym2 = js == 2 ? y0 : spare[(js + 0) % 3];   // (js - 3) mod 3
            if (act_b) {
                for (int k = 0; k < pz; ++k) {
                    const int o = sb.at(k, j, i);
                    const float cc = sm[ym1 + o];
                    const float Lf = lap_at(sm + ym1, sb, k, j, i, hx, hy, hz) - sm[F + o];
                    float v;
                    if (js == 1) {
                        const float z = p.tau * Lf;
                        v = cc + p.mut1 * z;
                        if (p.order == 2) sm[Z + o] = z;
                    } else {
                        v = p.mu[js] * cc + p.nu[js] * sm[ym2 + o] + p.mut_tau[js] * Lf;
                        if (p.order == 2) v = v + p.c0[js] * sm[y0 + o] + p.gt[js] * sm[Z + o];
                    }
                    put(c, sm, out, sb, k, j, i, v);
                }
            }
            c.cl.sync();
        }
        // the stage-s buffer becomes the iterate; the old iterate joins the spares
        const int last = (p.s - 1) % 3;
        const int ne = spare[last];
        spare[last] = y0;
        e = ne;
    };
    for (int n = 0; n < p.n_pre; ++n) superstep();

    // ---- r_B = f_B - L e_B, restricted by the 8-child mean into f_C
    if (act_b)
        for (int k = 0; k < pz; ++k) {
            const int o = sb.at(k, j, i);
            sm[Z + o] = sm[F + o] - lap_at(sm + e, sb, k, j, i, hx, hy, hz);
        }
    __syncthreads();
    float csum = 0.0f;
    if (act_c)
        for (int K = 0; K < cpz; ++K) {
            float pl[2];
            for (int a = 0; a < 2; ++a) {
                const float* r = sm + Z;
                const int k = 2 * K + a;
                const float r0 = r[sb.at(k, 2 * J, 2 * I)], r1 = r[sb.at(k, 2 * J, 2 * I + 1)];
                const float r4 = r[sb.at(k, 2 * J + 1, 2 * I)], r5 = r[sb.at(k, 2 * J + 1, 2 * I + 1)];
                pl[a] = (r0 + r1) + (r4 + r5);
            }
            const float cv = (pl[0] + pl[1]) * 0.125f;
            sm[FC + sc.at(K, J, I)] = cv;
            csum += cv;
        }
    if (p.remove_mean) {
        const float total = cluster_sum(c, sm, CRED, round, csum, red);
        const float mean = total / float(cnx * cny * (nz / 2));
        if (act_c)
            for (int K = 0; K < cpz; ++K) sm[FC + sc.at(K, J, I)] -= mean;
    }
    __syncthreads();

    // ---- coarsest level: accelerated RKL1 from e_C = 0 (App. A.5)
    const float chx = p.chx, chy = p.chy, chz = p.chz, tu = p.tau_unit;
    int y_cur = YC, y_prev = YC + fc, y_free = YC + 2 * fc;
    float f2 = 0.0f;
    if (act_c)
        for (int K = 0; K < cpz; ++K) {
            const float v = sm[FC + sc.at(K, J, I)];
            f2 = fmaf(v, v, f2);
        }
    const float r0sq = cluster_sum(c, sm, CRED, round, f2, red);
    const float tolsq = p.tol * p.tol * r0sq;
    int done = 0;
    for (int ss = 0; ss < p.max_ss; ++ss) {
        if (p.tol > 0.0f) {
            float acc = 0.0f;
            if (act_c)
                for (int K = 0; K < cpz; ++K) {
                    const float r = sm[FC + sc.at(K, J, I)] - lap_at(sm + y_cur, sc, K, J, I, chx, chy, chz);
                    acc = fmaf(r, r, acc);
                }
            if (cluster_sum(c, sm, CRED, round, acc, red) <= tolsq) break;
        }
        const int s = p.sched[ss];
        for (int js = 1; js <= s; ++js) {
            const float inv = 1.0f / float(js);
            const float mu = 2.0f - inv, nu = inv - 1.0f;
            const float mut = mu * tu;
            if (act_c)
                for (int K = 0; K < cpz; ++K) {
                    const int o = sc.at(K, J, I);
                    const float cc = sm[y_cur + o];
                    const float L = lap_at(sm + y_cur, sc, K, J, I, chx, chy, chz);
                    const float f = sm[FC + o];
                    const float v = js == 1 ? cc + tu * (L - f) : mu * cc + nu * sm[y_prev + o] + mut * (L - f);
                    put(c, sm, y_free, sc, K, J, I, v);
                }
            c.cl.sync();
            const int t = y_free;
            y_free = y_prev;
            y_prev = y_cur;
            y_cur = t;
        }
        ++done;
    }
    if (c.rank == 0 && tid == 0 && p.ss_done) *p.ss_done = done;

    // ---- e_B += P e_C (27/9/3/1 weights / 64).  The x / y ghosts of every
    // plane of e_C (z ghost planes included, their edges and corners too) are
    // set from the plane's interior by the boundary rule first.
    {
        const int gw = cnx + 2, gh = cny + 2, ng = 2 * gw + 2 * cny;     // ghost cells of one plane
        for (int t = tid; t < ng * (cpz + 2); t += blockDim.x) {
            const int K = t / ng - 1, g = t % ng;
            int gi, gj;
            if (g < gw) { gi = g - 1; gj = -1; }
            else if (g < 2 * gw) { gi = g - gw - 1; gj = cny; }
            else if (g < 2 * gw + cny) { gi = -1; gj = g - 2 * gw; }
            else { gi = cnx; gj = g - 2 * gw - cny; }
            (void)gh;
            int si = gi, sj = gj;
            float sg = 1.0f;
            if (gi < 0) { si = c.px ? cnx - 1 : 0; if (!c.px) sg = -sg; }
            else if (gi >= cnx) { si = c.px ? 0 : cnx - 1; if (!c.px) sg = -sg; }
            if (gj < 0) { sj = c.py ? cny - 1 : 0; if (!c.py) sg = -sg; }
            else if (gj >= cny) { sj = c.py ? 0 : cny - 1; if (!c.py) sg = -sg; }
            sm[y_cur + sc.at(K, gj, gi)] = sg * sm[y_cur + sc.at(K, sj, si)];
        }
    }
    __syncthreads();
    if (act_b) {
        const int Ia = i >> 1, Ja = j >> 1;
        const int Ib = Ia + ((i & 1) ? 1 : -1), Jb = Ja + ((j & 1) ? 1 : -1);
        const float* ec = sm + y_cur;
        auto q = [&](int K) {
            return 9.0f * ec[sc.at(K, Ja, Ia)] + 3.0f * ec[sc.at(K, Ja, Ib)] + 3.0f * ec[sc.at(K, Jb, Ia)] +
                   ec[sc.at(K, Jb, Ib)];
        };
        const float w = 1.0f / 64.0f;
        for (int k = 0; k < pz; k += 2) {
            const int K = k >> 1;
            const float qm = q(K - 1), q0 = q(K), qp = q(K + 1);
            const int o0 = sb.at(k, j, i), o1 = sb.at(k + 1, j, i);
            put(c, sm, e, sb, k, j, i, sm[e + o0] + (3.0f * q0 + qm) * w);
            put(c, sm, e, sb, k + 1, j, i, sm[e + o1] + (3.0f * q0 + qp) * w);
        }
    }
    c.cl.sync();

    for (int n = 0; n < p.n_post; ++n) superstep();

    if (act_b)
        for (int k = 0; k < pz; ++k) p.u_out[((size_t)(c.rank * pz + k) * ny + j) * nx + i] = sm[e + sb.at(k, j, i)];
    c.cl.sync();                                  // peers may still write this CTA's ghosts until here
}

size_t bottom_bytes(int nx, int ny, int nz, int nc) {
    const int pz = nz / nc;
    const size_t fb = (size_t)(nx + 2) * (ny + 2) * (pz + 2);
    const size_t fc = (size_t)(nx / 2 + 2) * (ny / 2 + 2) * (pz / 2 + 2);
    return (6 * fb + 4 * fc + 2 * kBottomMaxNC) * sizeof(float);
}

// Plans by level-B shape, filled before any graph capture (the occupancy query
// is not a stream operation, but it is kept out of captured code all the same).
struct BottomPlan {
    int nx, ny, nz, nc, threads;
    size_t bytes;
};
constexpr int kPlanCache = 64;
BottomPlan g_plans[kPlanCache];
int g_nplans = 0;
bool g_bottom_configured = false;

}  // namespace

cudaError_t bottom_configure() {
    if (g_bottom_configured) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_bottom_levels, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemLimit);
    if (e != cudaSuccess) return e;
    g_bottom_configured = true;
    return cudaSuccess;
}

// Cluster size for level B (nx, ny, nz): the largest power of two <= 8 that
// cuts nz into slabs of an even number of planes, with the fields in shared
// memory and one cluster of that size schedulable; 0 if none.
int bottom_plan(int nx, int ny, int nz, int s, int* threads, size_t* bytes) {
    if (s < 1 || s > kBottomMaxS || nx * ny > 1024 || nx % 2 || ny % 2 || nz % 2 || nx < 2 || ny < 2) return 0;
    for (int k = 0; k < g_nplans; ++k)
        if (g_plans[k].nx == nx && g_plans[k].ny == ny && g_plans[k].nz == nz) {
            *threads = g_plans[k].threads;
            *bytes = g_plans[k].bytes;
            return g_plans[k].nc;
        }
    int found = 0;
    const int th = ((nx * ny + 31) / 32) * 32;
    size_t by = 0;
    for (int nc = kBottomMaxNC; nc >= 1 && !found; nc >>= 1) {
        if (nz % (2 * nc)) continue;
        by = bottom_bytes(nx, ny, nz, nc);
        if (by > kSmemLimit) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nc);
        cfg.blockDim = dim3(th);
        cfg.dynamicSmemBytes = by;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = nc;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_bottom_levels, &cfg) == cudaSuccess && n > 0) found = nc;
        else cudaGetLastError();
    }
    if (g_nplans < kPlanCache) g_plans[g_nplans++] = BottomPlan{nx, ny, nz, found, th, by};
    *threads = th;
    *bytes = by;
    return found;
}

cudaError_t launch_bottom(const BottomParams& p, int nc, int threads, size_t bytes, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_bottom_levels, p);
}

}  // namespace sg
