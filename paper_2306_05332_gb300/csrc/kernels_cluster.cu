// The two coarsest levels of the FP32 V-cycle in one launch (Sec. 2.1 steps
// 2c-2e and 3, Eq. RKL_intermediate_source, App. A.5): a thread-block cluster
// holds level B (the second coarsest) in distributed shared memory and level
// C = B + 1 (the coarsest) whole in every CTA, and runs, without touching
// global memory between them,
//   the n_pre smoothing super-steps of B from e_B = 0,
//   r_B = f_B - L e_B and its 8-child restriction f_C (mean removed when every
//   axis is periodic, Eq. source_modification),
//   the accelerated RKL1 solve of L e_C = f_C from e_C = 0 (schedule s_k,
//   stopped by the coarse tolerance),
//   e_B += P e_C (27/9/3/1 prolongation) and the n_post smoothing super-steps.
//
// Level B.  CTA `rank` of the cluster owns the z slab [rank pz, (rank + 1) pz)
// of level B; every field is stored with a one-cell ghost layer.  A thread
// owns one (x, y) column of the slab.  Ghosts follow the boundary rule of the
// level (Eq. error_ghost: ghost = -active; Eq. periodic: the opposite cell):
// the thread writing a boundary cell writes the x / y ghost in its own CTA and
// the z ghost plane of the neighbouring CTA (through distributed shared
// memory), and a cluster barrier (release / acquire) ends every stage.
//
// Level C.  The restriction sends f_C to every CTA, and each CTA then solves
// the whole level by itself with one block barrier per stage: the same
// arithmetic on the same data, so every CTA holds the same e_C, takes the same
// stop decision (block sums in a fixed order) and has every coarse plane its
// prolongation needs.  The solve works on strips of four x cells in dense
// rotating buffers, each neighbour strip picked by the boundary rule, in the
// shared memory the level-B stage buffers free meanwhile.
//
// The arithmetic of every stage, of the residual, the restriction and the
// prolongation is written in the order of the single-level kernels.
#include "sg_internal.cuh"

#include <cooperative_groups.h>

#include <mutex>

namespace cg = cooperative_groups;

namespace sg {

namespace {

constexpr int kBottomMaxNC = 16;         // CTAs per cluster (16: a non-portable size, where the device allows it)
constexpr size_t kSmemLimit = 227u * 1024u - 1024u;   // dynamic shared memory per CTA

__device__ __forceinline__ float lap7f(float c, float xm, float xp, float ym, float yp, float zm, float zp, float hx,
                                       float hy, float hz) {
    const float two_c = 2.0f * c;
    return ((xm - two_c) + xp) * hx + ((ym - two_c) + yp) * hy + ((zm - two_c) + zp) * hz;
}

// A field of level B: (pz + 2) planes of (ny + 2) rows of nx + 8 floats, the
// interior of a row at offset 4 (4-cell strips are 16-byte aligned) and its x
// ghosts at offsets 3 and nx + 4.
struct Slab {
    int nx, ny, pz, row, plane;
    __device__ int at(int k, int j, int i) const { return (k + 1) * plane + (j + 1) * row + 4 + i; }
};

__device__ __forceinline__ Slab make_slab(int nx, int ny, int pz) {
    Slab s;
    s.nx = nx;
    s.ny = ny;
    s.pz = pz;
    s.row = nx + 8;
    s.plane = (nx + 8) * (ny + 2);
    return s;
}

struct Ctx {
    cg::cluster_group cl;
    int rank, nc;
    bool px, py, pz;
};

__device__ __forceinline__ float4 ld4b(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4b(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 negb(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// The strip of cells 4q .. 4q + 3 of row j, plane k of field `f`, with its
// ghosts as put() writes them for single cells.
__device__ __forceinline__ void put4(const Ctx& c, float* sm, int f, const Slab& s, int k, int j, int q, float4 v) {
    float* fl = sm + f;
    const int o = s.at(k, j, 4 * q);
    st4b(fl + o, v);
    if (q == 0) fl[c.px ? s.at(k, j, s.nx) : o - 1] = c.px ? v.x : -v.x;
    if (4 * q + 4 == s.nx) fl[c.px ? s.at(k, j, -1) : o + 4] = c.px ? v.w : -v.w;
    if (j == 0) st4b(fl + s.at(k, c.py ? s.ny : -1, 4 * q), c.py ? v : negb(v));
    if (j == s.ny - 1) st4b(fl + s.at(k, c.py ? -1 : s.ny, 4 * q), c.py ? v : negb(v));
    if (k == 0) {
        if (c.rank > 0 || c.pz) {
            const int peer = c.rank > 0 ? c.rank - 1 : c.nc - 1;
            st4b(c.cl.map_shared_rank(sm, peer) + f + s.at(s.pz, j, 4 * q), v);
        } else {
            st4b(fl + s.at(-1, j, 4 * q), negb(v));
        }
    }
    if (k == s.pz - 1) {
        if (c.rank < c.nc - 1 || c.pz) {
            const int peer = c.rank < c.nc - 1 ? c.rank + 1 : 0;
            st4b(c.cl.map_shared_rank(sm, peer) + f + s.at(-1, j, 4 * q), v);
        } else {
            st4b(fl + s.at(s.pz, j, 4 * q), negb(v));
        }
    }
}

// L of the strip at offset o of field y (cell by cell as lap_at).
__device__ __forceinline__ float4 lap4b(const float* y, const Slab& s, int o, float hx, float hy, float hz) {
    const float4 cc = ld4b(y + o), ym = ld4b(y + o - s.row), yp = ld4b(y + o + s.row);
    const float4 zm = ld4b(y + o - s.plane), zp = ld4b(y + o + s.plane);
    const float xl = y[o - 1], xr = y[o + 4];
    return make_float4(lap7f(cc.x, xl, cc.y, ym.x, yp.x, zm.x, zp.x, hx, hy, hz),
                       lap7f(cc.y, cc.x, cc.z, ym.y, yp.y, zm.y, zp.y, hx, hy, hz),
                       lap7f(cc.z, cc.y, cc.w, ym.z, yp.z, zm.z, zp.z, hx, hy, hz),
                       lap7f(cc.w, cc.z, xr, ym.w, yp.w, zm.w, zp.w, hx, hy, hz));
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

// Level C held whole with a ghost layer on every face (for the prolongation).
struct Full {
    int nx, ny, nz, row, plane;
    __device__ int at(int k, int j, int i) const { return (k + 1) * plane + (j + 1) * row + (i + 1); }
};

// Packed FP32 pairs (f32x2): two independent FP32 operations per instruction,
// each rounded as the scalar one.
__device__ __forceinline__ unsigned long long pk2(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 fma2f(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
    return upk2(d);
}
__device__ __forceinline__ float2 add2f(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
__device__ __forceinline__ float2 mul2f(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
__device__ __forceinline__ float2 lo2f(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2f(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 dupf(float a) { return make_float2(a, a); }

__device__ __forceinline__ float4 ld4s(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4s(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 neg4(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

__global__ void __launch_bounds__(1024) k_bottom_levels(const __grid_constant__ BottomParams p) {
    extern __shared__ __align__(16) float sm[];
    __shared__ float red[32];
    Ctx c{cg::this_cluster(), 0, 0, p.per[0] != 0, p.per[1] != 0, p.per[2] != 0};
    c.rank = (int)c.cl.block_rank();
    c.nc = (int)c.cl.num_blocks();
    const int nx = p.nx, ny = p.ny, nz = p.nz, pz = nz / c.nc;
    const int cnx = nx / 2, cny = ny / 2, cnz = nz / 2, cpz = pz / 2;
    const int ncc = cnx * cny * cnz;                 // cells of level C
    const Slab sb = make_slab(nx, ny, pz);
    Full sf;
    sf.nx = cnx;
    sf.ny = cny;
    sf.nz = cnz;
    sf.row = cnx + 2;
    sf.plane = (cnx + 2) * (cny + 2);
    const int fb = sb.plane * (pz + 2);
    // level B: rhs F, iterate E, then a region U of four slab fields (Z0 /
    // residual and three stage buffers) that holds level C's three iterates
    // and its ghosted copy while level C is solved; FC: level C's rhs, dense
    const int F = 0, E = fb, U = 2 * fb, FC = 6 * fb;
    const int nfl = FC + ncc;
    const int tid = threadIdx.x;
    const bool act_c = tid < cnx * cny;
    const int I = act_c ? tid % cnx : 0, J = act_c ? tid / cnx : 0;
    const float hx = p.hx, hy = p.hy, hz = p.hz;
    // level B by strips of four x cells: strip t is (q, j, k) = (t % nq, t / nq % ny,
    // t / (nq ny)); a thread owns strips tid and tid + blockDim (the plan keeps
    // nq ny pz <= 2 blockDim)
    const int nqb = nx >> 2, nsb = nqb * ny * pz;
    int sq_[2], sj_[2], sk_[2], so_[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int t = min(tid + a * (int)blockDim.x, nsb - 1);
        sq_[a] = t % nqb;
        sj_[a] = (t / nqb) % ny;
        sk_[a] = t / (nqb * ny);
        so_[a] = sb.at(sk_[a], sj_[a], 4 * sq_[a]);
    }
    const int ns = tid < nsb ? (tid + (int)blockDim.x < nsb ? 2 : 1) : 0;

    for (int t = tid; t < nfl; t += blockDim.x) sm[t] = 0.0f;
    c.cl.sync();                                 // no peer writes a ghost before it is cleared
#pragma unroll
    for (int a = 0; a < 2; ++a)
        if (a < ns) st4b(sm + F + so_[a],
             ld4b(p.rhs + ((size_t)(c.rank * pz + sk_[a]) * ny + sj_[a]) * nx + 4 * sq_[a]));
    __syncthreads();

    // ---- smoothing super-steps of level B (App. A, Eq. RKL_intermediate_source)
    const int Z = U;
    int e = E;                                    // current iterate (zero)
    int spare[3] = {U + fb, U + 2 * fb, U + 3 * fb};
    auto superstep = [&]() {
        const int y0 = e;
        for (int js = 1; js <= p.s; ++js) {
            const int out = spare[(js - 1) % 3];
            const int ym1 = js == 1 ? y0 : spare[(js - 2) % 3];
            const int ym2 = js == 2 ? y0 : spare[js % 3];         // (js - 3) mod 3
#pragma unroll
        #pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (a >= ns) break;
                const int o = so_[a];
                const float4 cc = ld4b(sm + ym1 + o), fv = ld4b(sm + F + o);
                const float4 L = lap4b(sm + ym1, sb, o, hx, hy, hz);
                const float cv[4] = {cc.x, cc.y, cc.z, cc.w}, lv[4] = {L.x, L.y, L.z, L.w};
                const float fw[4] = {fv.x, fv.y, fv.z, fv.w};
                float v[4];
                if (js == 1) {
                    float zz[4];
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        const float Lf = lv[e2] - fw[e2];
                        zz[e2] = p.tau * Lf;
                        v[e2] = cv[e2] + p.mut1 * zz[e2];
                    }
                    if (p.order == 2) st4b(sm + Z + o, make_float4(zz[0], zz[1], zz[2], zz[3]));
                } else {
                    const float4 pm = ld4b(sm + ym2 + o);
                    const float pv[4] = {pm.x, pm.y, pm.z, pm.w};
                    float yv[4] = {0.f, 0.f, 0.f, 0.f}, zv[4] = {0.f, 0.f, 0.f, 0.f};
                    if (p.order == 2) {
                        const float4 y4 = ld4b(sm + y0 + o), z4 = ld4b(sm + Z + o);
                        yv[0] = y4.x; yv[1] = y4.y; yv[2] = y4.z; yv[3] = y4.w;
                        zv[0] = z4.x; zv[1] = z4.y; zv[2] = z4.z; zv[3] = z4.w;
                    }
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        const float Lf = lv[e2] - fw[e2];
                        v[e2] = p.mu[js] * cv[e2] + p.nu[js] * pv[e2] + p.mut_tau[js] * Lf;
                        if (p.order == 2) v[e2] = v[e2] + p.c0[js] * yv[e2] + p.gt[js] * zv[e2];
                    }
                }
                put4(c, sm, out, sb, sk_[a], sj_[a], sq_[a], make_float4(v[0], v[1], v[2], v[3]));
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
    // the iterate back to its home E (ghost planes included), so that U is free
    if (e != E) {
        for (int t = tid; t < fb; t += blockDim.x) sm[E + t] = sm[e + t];
        for (int k = 0; k < 3; ++k)
            if (spare[k] == E) spare[k] = e;
        e = E;
        __syncthreads();
    }

    // ---- r_B = f_B - L e_B, restricted by the 8-child mean into f_C, which
    // every CTA receives whole
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (a >= ns) break;
        const int o = so_[a];
        const float4 fv = ld4b(sm + F + o), L = lap4b(sm + e, sb, o, hx, hy, hz);
        st4b(sm + Z + o, make_float4(fv.x - L.x, fv.y - L.y, fv.z - L.z, fv.w - L.w));
    }
    __syncthreads();
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
            const int o = FC + ((c.rank * cpz + K) * cny + J) * cnx + I;
            for (int q = 0; q < c.nc; ++q) c.cl.map_shared_rank(sm, q)[o] = cv;
        }
    c.cl.sync();

    // ---- level C, whole in every CTA: the same arithmetic on the same data in
    // each, so all CTAs hold the same e_C and take the same steps (accelerated
    // RKL1 from e_C = 0, App. A.5).  Strips of four x cells; the boundary rule
    // picks each neighbour strip.
    const float chx = p.chx, chy = p.chy, chz = p.chz, tu = p.tau_unit;
    if (p.remove_mean) {                         // Eq. source_modification on level C
        float s = 0.0f;
        for (int t = tid; t < ncc; t += blockDim.x) s += sm[FC + t];
        const float mean = block_sum(s, red) / float(ncc);
        for (int t = tid; t < ncc; t += blockDim.x) sm[FC + t] -= mean;
        __syncthreads();
    }
    // one strip of four x cells per thread (the plan guarantees enough
    // threads); its iterate, previous iterate and f stay in registers, and
    // every stage publishes the new iterate in one of two dense buffers
    const int nq = cnx >> 2, nrow = nq * cny, nstrip = nrow * cnz;
    const bool own = tid < nstrip;
    const int q = own ? tid % nq : 0, jj = own ? (tid / nq) % cny : 0, kk = own ? tid / nrow : 0;
    // neighbour strips (float4 index) and x cells (float index); -1: the
    // Dirichlet reflection of this strip's own value
    const int oym = jj > 0 ? tid - nq : (c.py ? tid + (cny - 1) * nq : -1);
    const int oyp = jj < cny - 1 ? tid + nq : (c.py ? tid - (cny - 1) * nq : -1);
    const int ozm = kk > 0 ? tid - nrow : (c.pz ? tid + (cnz - 1) * nrow : -1);
    const int ozp = kk < cnz - 1 ? tid + nrow : (c.pz ? tid - (cnz - 1) * nrow : -1);
    const int oxl = q > 0 ? 4 * tid - 1 : (c.px ? 4 * (tid + nq - 1) + 3 : -1);
    const int oxr = q < nq - 1 ? 4 * tid + 4 : (c.px ? 4 * (tid - nq + 1) : -1);
    int pub = U;                                   // buffer holding every strip's current iterate
    const int other = U + ncc;
    for (int t = tid; t < 2 * ncc; t += blockDim.x) sm[U + t] = 0.0f;
    const float4 f = own ? ld4s(sm + FC + 4 * tid) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 cur = make_float4(0.f, 0.f, 0.f, 0.f), prev = cur;
    const float f2 = own ? fmaf(f.x, f.x, fmaf(f.y, f.y, fmaf(f.z, f.z, f.w * f.w))) : 0.0f;
    const float r0sq = block_sum(f2, red);       // (its barriers also order the writes above)
    const float tolsq = p.tol * p.tol * r0sq;
    // L of the thread's strip as two packed pairs: h_x (x neighbours) +
    // h_y (y neighbours) + h_z (z neighbours) - 2 (h_x + h_y + h_z) c
    const float2 hx2 = dupf(chx), hy2 = dupf(chy), hz2 = dupf(chz), md2 = dupf(-2.0f * (chx + chy + chz));
    const float2 nf01 = make_float2(-f.x, -f.y), nf23 = make_float2(-f.z, -f.w);
    auto lap_minus_f = [&](const float* y, float2& d01, float2& d23) {     // L cur - f
        const float4 ym = oym >= 0 ? ld4s(y + 4 * oym) : neg4(cur);
        const float4 yp = oyp >= 0 ? ld4s(y + 4 * oyp) : neg4(cur);
        const float4 zm = ozm >= 0 ? ld4s(y + 4 * ozm) : neg4(cur);
        const float4 zp = ozp >= 0 ? ld4s(y + 4 * ozp) : neg4(cur);
        const float xl = oxl >= 0 ? y[oxl] : -cur.x;
        const float xr = oxr >= 0 ? y[oxr] : -cur.w;
        const float4 cc = cur;
        const float2 sx01 = add2f(make_float2(xl, cc.x), make_float2(cc.y, cc.z));
        const float2 sx23 = add2f(make_float2(cc.y, cc.z), make_float2(cc.w, xr));
        const float2 L01 = fma2f(hx2, sx01, fma2f(hy2, add2f(lo2f(ym), lo2f(yp)),
                                                  fma2f(hz2, add2f(lo2f(zm), lo2f(zp)), mul2f(md2, lo2f(cc)))));
        const float2 L23 = fma2f(hx2, sx23, fma2f(hy2, add2f(hi2f(ym), hi2f(yp)),
                                                  fma2f(hz2, add2f(hi2f(zm), hi2f(zp)), mul2f(md2, hi2f(cc)))));
        d01 = add2f(L01, nf01);
        d23 = add2f(L23, nf23);
    };
    int done = 0;
    for (int ss = 0; ss < p.max_ss; ++ss) {
        if (p.tol > 0.0f) {
            float acc = 0.0f;
            if (own) {
                float2 d01, d23;
                lap_minus_f(sm + pub, d01, d23);
                acc = fmaf(d01.x, d01.x, fmaf(d01.y, d01.y, fmaf(d23.x, d23.x, d23.y * d23.y)));
            }
            if (block_sum(acc, red) <= tolsq) break;
        }
        const int s = p.sched[ss];
        for (int js = 1; js <= s; ++js) {
            const float inv = 1.0f / float(js);
            const float mu = 2.0f - inv, nu = inv - 1.0f;
            const int dst = pub == U ? other : U;
            if (own) {
                float2 d01, d23;
                lap_minus_f(sm + pub, d01, d23);
                const float4 cc = cur;
                float2 v01, v23;
                if (js == 1) {                     // Y1 = Y0 + tau_unit (L Y0 - f)
                    v01 = fma2f(dupf(tu), d01, lo2f(cc));
                    v23 = fma2f(dupf(tu), d23, hi2f(cc));
                } else {                           // Y_j = mu Y_{j-1} + nu Y_{j-2} + mu tau_unit (L Y_{j-1} - f)
                    const float2 mu2 = dupf(mu), nu2 = dupf(nu), mt2 = dupf(mu * tu);
                    v01 = fma2f(mt2, d01, fma2f(nu2, lo2f(prev), mul2f(mu2, lo2f(cc))));
                    v23 = fma2f(mt2, d23, fma2f(nu2, hi2f(prev), mul2f(mu2, hi2f(cc))));
                }
                prev = cc;
                cur = make_float4(v01.x, v01.y, v23.x, v23.y);
                st4s(sm + dst + 4 * tid, cur);
            }
            __syncthreads();
            pub = dst;
        }
        ++done;
    }
    if (c.rank == 0 && tid == 0 && p.ss_done) *p.ss_done = done;
    const int y_cur = pub;

    // ---- e_B += P e_C (27/9/3/1 weights / 64) from a ghosted copy of e_C:
    // every ghost (edges and corners too) set by the boundary rule
    const int EC = U + 3 * ncc;
    const int ff = sf.plane * (cnz + 2);
    for (int t = tid; t < ff; t += blockDim.x) {
        const int gk = t / sf.plane - 1, gj = (t / sf.row) % (cny + 2) - 1, gi = t % sf.row - 1;
        float sg = 1.0f;
        auto mapc = [&](int v, int n, bool per) {
            if (v < 0) { if (!per) sg = -sg; return per ? n - 1 : 0; }
            if (v >= n) { if (!per) sg = -sg; return per ? 0 : n - 1; }
            return v;
        };
        const int si = mapc(gi, cnx, c.px), sj = mapc(gj, cny, c.py), sk = mapc(gk, cnz, c.pz);
        sm[EC + t] = sg * sm[y_cur + (sk * cny + sj) * cnx + si];
    }
    __syncthreads();
    {
        const float* ec = sm + EC;
        const float w = 1.0f / 64.0f;
    #pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (a >= ns) break;
            const int j = sj_[a], kk = c.rank * pz + sk_[a];
            const int Ja = j >> 1, Jb = Ja + ((j & 1) ? 1 : -1);
            const int K = kk >> 1, Ko = (kk & 1) ? K + 1 : K - 1;     // parent plane, the other one
            const float4 old = ld4b(sm + e + so_[a]);
            const float ov[4] = {old.x, old.y, old.z, old.w};
            float v[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
                const int i = 4 * sq_[a] + e2;
                const int Ia = i >> 1, Ib = Ia + ((i & 1) ? 1 : -1);
                const float q0 = 9.0f * ec[sf.at(K, Ja, Ia)] + 3.0f * ec[sf.at(K, Ja, Ib)] +
                                 3.0f * ec[sf.at(K, Jb, Ia)] + ec[sf.at(K, Jb, Ib)];
                const float qo = 9.0f * ec[sf.at(Ko, Ja, Ia)] + 3.0f * ec[sf.at(Ko, Ja, Ib)] +
                                 3.0f * ec[sf.at(Ko, Jb, Ia)] + ec[sf.at(Ko, Jb, Ib)];
                v[e2] = ov[e2] + (3.0f * q0 + qo) * w;
            }
            put4(c, sm, e, sb, sk_[a], j, sq_[a], make_float4(v[0], v[1], v[2], v[3]));
        }
    }
    c.cl.sync();

    for (int n = 0; n < p.n_post; ++n) superstep();

#pragma unroll
    for (int a = 0; a < 2; ++a)
        if (a < ns) st4b(p.u_out + ((size_t)(c.rank * pz + sk_[a]) * ny + sj_[a]) * nx + 4 * sq_[a], ld4b(sm + e + so_[a]));
    c.cl.sync();                                  // peers may still write this CTA's ghosts until here
}

// Shared memory of one CTA, or 0 where level C does not split into 4-cell
// strips, has more strips than the CTA has threads, level B has more strips
// than twice the threads, or level C does not fit (two dense iterates and a
// ghosted copy) in the region of four level-B slab fields.
size_t bottom_bytes(int nx, int ny, int nz, int nc) {
    const int pz = nz / nc;
    const size_t fb = (size_t)(nx + 8) * (ny + 2) * (pz + 2);
    const size_t ncc = (size_t)(nx / 2) * (ny / 2) * (nz / 2);
    const size_t ff = (size_t)(nx / 2 + 2) * (ny / 2 + 2) * (nz / 2 + 2);
    const size_t threads = ((size_t)nx * ny + 31) / 32 * 32;
    const size_t strips_b = (size_t)(nx / 4) * ny * pz;
    if ((nx / 2) % 4 != 0 || ncc / 4 > threads || strips_b > 2 * threads || 3 * ncc + ff > 4 * fb) return 0;
    return (6 * fb + ncc) * sizeof(float);
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
std::mutex g_plans_mu;          // the cache and the one-time configuration, for callers on several threads

}  // namespace

cudaError_t bottom_configure() {
    std::lock_guard<std::mutex> lock(g_plans_mu);
    if (g_bottom_configured) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_bottom_levels, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemLimit);
    if (e != cudaSuccess) return e;
    // clusters of 16 CTAs are opt-in; where the device refuses, the plan below
    // finds no schedulable cluster of 16 and takes 8
    if (cudaFuncSetAttribute(k_bottom_levels, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    g_bottom_configured = true;
    return cudaSuccess;
}

// Cluster size for level B (nx, ny, nz): the largest power of two <= 16 that
// cuts nz into slabs of an even number of planes, with the fields in shared
// memory and one cluster of that size schedulable; 0 if none.
int bottom_plan(int nx, int ny, int nz, int s, int* threads, size_t* bytes) {
    if (s < 1 || s > kBottomMaxS || nx * ny > 1024 || nx % 2 || ny % 2 || nz % 2 || nx < 2 || ny < 2) return 0;
    std::lock_guard<std::mutex> lock(g_plans_mu);
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
        if (by == 0 || by > kSmemLimit) continue;
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
