// Fused RKL super-step for s = 2 and 3 stages (App. A, Eq.
// RKL_intermediate_source): all stages in one pass over HBM, FP32, for the
// error equation of the mixed-precision V-cycle (homogeneous Dirichlet or
// periodic ghosts).
//
// Work split.  A CTA owns a TX x TY column of the level (TX = 64 for s = 3
// with a general Y0, 32 otherwise; TY = 16 or 14), widened by a halo (4 cells
// in x, s cells in y), and streams it along z.  Stage j is computed on the
// tile widened by s - j cells in strips of four x cells; every thread owns the
// two strips of one row pair of ONE stage for the whole stream, and each
// stage's row pairs fill whole warps.  In phase t, stage j works on plane
// t - (2j - 1): it reads only planes finished in earlier phases, so one
// barrier per phase suffices.
//
// Boundaries without branches.  For a Dirichlet axis the halo outside the box
// is loaded as the odd reflection of the interior (cell -1-k holds -cell k,
// repeated with period 2n), for a periodic axis as the periodic image.  The
// 7-point stencil and the stage recurrence commute with that reflection
// exactly (negation and operand order are exact in IEEE arithmetic), so every
// stage computes the odd extension of the solution and the ghost rule of Eq.
// error_ghost (ghost = -active) holds at the walls with no per-cell test.
// Loads arrive by cp.async; a thread negates the reflected cells it loaded.
//
// Shared-memory traffic.  A thread keeps its strip of the planes p - 1 and p
// of its input stage in registers (it reads plane p + 1 as it walks z), takes
// its x neighbours from the adjacent lanes by shuffles, and reads only the
// y neighbours and one combined source field from shared memory.  The first
// stage folds everything later stages take from Y0, Z0 = tau (L Y0 - f), f and
// Y1 into one field per stage:
//   Y_j = mu_j Y_{j-1} + mu~_j tau L Y_{j-1} + W_j,
//   W_j = nu_j Y_{j-2} + c0_j Y0 + gamma~_j Z0 - mu~_j tau f   (RKL1: c0 = gamma~ = 0)
// and with Y0 = 0 every W_j is a multiple of f.  So is Y1 = -mu~_1 tau f then:
// the pipeline starts at stage 2, a stencil of f with that factor folded into
// its coefficients, and runs s - 1 stencil stages on a halo of s - 1 cells.
//
// Ring depths are powers of two (a slot is a mask of the phase index), and the
// phase loop is unrolled by three so that the z window rotates by register
// renaming.  A launch cuts every tile into the same z chunks, so neighbouring
// tiles stream the same planes at about the same time and share halos in L2.
//
// Latency.  Planes are staged into shared memory two phases before their
// first use (staging four phases ahead measured no faster).  A phase issues
// its copies at its end, after its own shared-memory reads: issued at the
// start of the phase they queued in the load/store pipeline ahead of every
// stage's loads (124.6 against 116.4 us per general 256^3 launch).
//
// HBM traffic per super-step: read Y0 + read f + write Y_s (12 B/cell; 8 B/cell
// when Y0 = 0).  Halo cells are re-read from L2 by neighbouring tiles.
#include "sg_internal.cuh"

#include <cuda.h>          // CUtensorMap and its encoder's signature (called through the runtime's entry point)

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <type_traits>

namespace sg {

namespace {

__device__ __forceinline__ void cpa4(float* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa16(float* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ---- TMA staging: box copies completing on an mbarrier ---------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Every wait is bounded: a phase that does not complete within kWaitTries
// hardware-suspended tries (seconds) is reported instead of hanging the GPU.
constexpr int kWaitTries = 1 << 22;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (int i = 0; i < kWaitTries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Generic-proxy accesses of a ring slot before the barrier that ends a phase,
// async-proxy (TMA) writes of the same slot after it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tma_load(float* dst, const CUtensorMap* map, int x, int y, int z,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_prefetch(const CUtensorMap* map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(map), "r"(x), "r"(y),
                 "r"(z)
                 : "memory");
}

// Bounded waits that gave up (a device counter the host reads when a solve
// turns non-finite; the kernel that gave up writes a NaN into its output).
__device__ unsigned int g_lean_wait_timeouts = 0;

// Index of cell v of an axis of n cells in the stored array and its sign:
// periodic image, or odd reflection about both walls (period 2n).
__host__ __device__ __forceinline__ int map_axis(int v, int n, bool periodic, int* sign) {
    if (v >= 0 && v < n) {                  // inside the box: no integer division
        *sign = 1;
        return v;
    }
    if (periodic) {
        *sign = 1;
        const int m = v % n;
        return m < 0 ? m + n : m;
    }
    int m = v % (2 * n);
    if (m < 0) m += 2 * n;
    if (m < n) {
        *sign = 1;
        return m;
    }
    *sign = -1;
    return 2 * n - 1 - m;
}

template <int S, bool ZERO, int TYV>
struct Lean {
    // pipeline stages: with Y0 = 0 the first RKL stage is Y1 = mu~_1 tau (-f),
    // so RKL stage 2 is a stencil of f itself and the pipeline runs stages
    // 2 .. s (pipeline stage j computes RKL stage j + 1)
    static constexpr int NS = ZERO ? S - 1 : S;
    // tile width: 64 cells for s = 3 with a general Y0 (one CTA of 15 - 16
    // warps per SM: less x halo per cell than two 32-wide CTAs, measured 124.6
    // against 132.6 us per 256^3 super-step), otherwise 32 (two or three
    // lighter CTAs per SM)
    static constexpr int TX = (ZERO || S < 3) ? 32 : 64, TY = TYV, HX = 4;
    static constexpr int W = TX + 2 * HX;            // plane row (floats)
    static constexpr int H = TY + 2 * NS;            // plane rows
    static constexpr int Q = W / 4;                  // strips per row
    // planes store the even rows, then the odd rows, so that the first rows of
    // consecutive row pairs are contiguous (conflict-free quarter-warp accesses);
    // each half starts on a 128-byte boundary, the alignment of a TMA box copy
    static constexpr int HO = ((H / 2) * W + 31) / 32 * 32;   // offset of the odd rows (floats)
    static constexpr int P = 2 * HO;                 // floats per plane
    static constexpr int HQ = H * Q;                 // strips per plane
    __host__ __device__ static constexpr int rowoff(int r) { return (r & 1) * HO + (r >> 1) * W; }
    // pipeline stage j covers rows [j, H - j) (an even count) and strips
    // [qlo(j), qhi(j)); one item = the strips of rows r and r + 1 at one q
    __host__ __device__ static constexpr int qlo(int j) { return (HX - (NS - j)) / 4; }
    __host__ __device__ static constexpr int qhi(int j) { return (HX + TX + (NS - j) + 3) / 4; }
    __host__ __device__ static constexpr int nq(int j) { return qhi(j) - qlo(j); }
    __host__ __device__ static constexpr int items(int j) { return j > NS ? 0 : nq(j) * ((H - 2 * j) / 2); }
    __host__ __device__ static constexpr int warps(int j) { return (items(j) + 31) / 32; }
    static constexpr int T2 = 32 * warps(1);         // first thread of pipeline stage 2 (or end)
    static constexpr int T3 = T2 + 32 * warps(2);    // first thread of pipeline stage 3 (or end)
    static constexpr int TS = T3 + 32 * warps(3);    // threads with stage work
    static constexpr int TL = 32 * ((HQ + 31) / 32); // threads [0, HQ) stage one strip of Y0 and of f
    static constexpr int NT = TS > TL ? TS : TL;
    // Registers per thread that let `ctas` CTAs share an SM: the register file
    // is split over four scheduler partitions of 16384 registers, a warp sits
    // on one partition and holds a multiple of 8 registers per thread.
    __host__ __device__ static constexpr int reg_cap(int ctas) {
        return (16384 / ((((ctas * NT / 32) + 3) / 4) * 32)) / 8 * 8;
    }
    // ring depths (planes, powers of two)
    static constexpr int RY0 = ZERO ? 0 : 4;         // Y0: p, p + 1 read, p + 2 in flight
    static constexpr int RF = ZERO ? 8 : 4;          // f (Y0 = 0: read by every stage, lag up to 2 NS - 1)
    static constexpr int RY = 4;                     // Y_j, j < NS
    static constexpr int RW2 = ZERO ? 0 : 4;         // W_2: written at lag 1, read at lag 3
    static constexpr int RW3 = (ZERO || S < 3) ? 0 : 8;   // W_3: written at lag 1, read at lag 5
    static constexpr int OY0 = 0;
    static constexpr int OF = OY0 + RY0 * P;
    static constexpr int OY = OF + RF * P;           // ring of pipeline stage j at OY + (j - 1) RY P
    static constexpr int OW2 = OY + (NS - 1) * RY * P;
    static constexpr int OW3 = OW2 + RW2 * P;
    static constexpr int NFLOATS = OW3 + RW3 * P;
    static constexpr int NBAR = 4;                   // TMA path: one mbarrier per plane in flight
    static constexpr size_t BYTES = size_t(NFLOATS) * sizeof(float) + NBAR * sizeof(unsigned long long);
    // CTAs per SM the registers are budgeted for: three for the light Y0 = 0
    // variant where that leaves at least 88 registers per thread, otherwise
    // two where the shared memory holds two, else one
    static constexpr int SMEM_CTAS = int((228u * 1024u) / (BYTES + 1024u));
    static constexpr int CTAS = (ZERO && reg_cap(3) >= 88) ? 3 : (SMEM_CTAS >= 2 ? 2 : 1);
    static_assert(S == 2 || S == 3, "lean super-step covers s = 2, 3");
    static_assert(HX >= NS - 1 && HX % 4 == 0, "x halo");
    static_assert(TY % 2 == 0 && H % 2 == 0, "row pairs");
    static_assert(!ZERO || RF >= 2 * NS + 2, "f ring spans the staged planes and the oldest read");
    static_assert(BYTES <= 227u * 1024u, "rings exceed the shared memory of one CTA");
    static_assert(NT <= 1024, "block size");
};

// Coefficients, all FP32 (the kernel never converts from FP64).
struct LeanCoef {
    float ax[4], ay[4], az[4], b[4];    // stage j >= 2: Y_j = ax sx + ay sy + az sz + b c + W_j
    float ihx2, ihy2, ihz2, m2s;        // stage 1: Lf = ihx2 sx + ihy2 sy + ihz2 sz + m2s c - f
    float m1t;                          //          Y1 = c + m1t Lf
    float k2y0, k2z, k2f;               //          W2 = k2y0 c + k2z Lf + k2f f
    float k3c, k3l, k3f;                //          W3 = nu_3 Y1 + c0_3 c + gamma~_3 tau Lf - mu~_3 tau f
                                        //             = k3c c + k3l Lf + k3f f  (Y1 = c + m1t Lf)
    float kz[4];                        // Y0 = 0: Y1 = kz[1] f, W_j = kz[j] f
    float zx, zy, zz, zb;               // Y0 = 0: Y2 = zx sx(f) + zy sy(f) + zz sz(f) + zb f
};

// Source of one 4-cell strip of a staged plane.
struct LoadDesc {
    int dst;        // offset in the plane (floats); -1: this thread loads nothing
    int row;        // source row offset (y index * nx)
    int x01, x23;   // source x of the four cells, 16 bits each
    int flags;      // bit 4: one 16-byte copy; bits 0-3: cells negated by the x/y reflection
};

__device__ __forceinline__ LoadDesc make_desc(int k, int X0, int Yt, const LevelGeom& g, bool vec_ok, int Q,
                                              int HO, int W) {
    LoadDesc d;
    const int r = k / Q, q = k % Q;
    d.dst = (r & 1) * HO + (r >> 1) * W + 4 * q;
    int sy;
    const int yy = map_axis(Yt + r, g.ny, g.per[1] != 0, &sy);
    d.row = yy * g.nx;
    int xs[4], mask = 0;
    bool contiguous = true;
    for (int e = 0; e < 4; ++e) {
        int sx;
        xs[e] = map_axis(X0 + 4 * q + e, g.nx, g.per[0] != 0, &sx);
        if (sx * sy < 0) mask |= 1 << e;
        if (sx < 0 || xs[e] != xs[0] + e) contiguous = false;
    }
    d.x01 = xs[0] | (xs[1] << 16);
    d.x23 = xs[2] | (xs[3] << 16);
    const bool vec = vec_ok && contiguous && (xs[0] & 3) == 0;
    d.flags = mask | (vec ? 16 : 0);
    return d;
}

__device__ __forceinline__ void issue(const LoadDesc& d, float* plane_dst, const float* plane_src) {
    if (d.dst < 0) return;
    const float* s = plane_src + d.row;
    if (d.flags & 16) {
        cpa16(plane_dst + d.dst, s + (d.x01 & 0xffff));
    } else {
        cpa4(plane_dst + d.dst + 0, s + (d.x01 & 0xffff));
        cpa4(plane_dst + d.dst + 1, s + (d.x01 >> 16));
        cpa4(plane_dst + d.dst + 2, s + (d.x23 & 0xffff));
        cpa4(plane_dst + d.dst + 3, s + (d.x23 >> 16));
    }
}

// After the thread's copies arrived: negate the cells whose reflection sign
// (x, y and the plane's z sign) is negative.
__device__ __forceinline__ void fixup(const LoadDesc& d, float* plane_dst, int zsign) {
    if (d.dst < 0) return;
    const int m = zsign < 0 ? (~d.flags & 15) : (d.flags & 15);
    if (m == 0) return;
    float4* p = reinterpret_cast<float4*>(plane_dst + d.dst);
    float4 v = *p;
    if (m & 1) v.x = -v.x;
    if (m & 2) v.y = -v.y;
    if (m & 4) v.z = -v.z;
    if (m & 8) v.w = -v.w;
    *p = v;
}

// TMA path, tiles that reach past a Dirichlet x or y wall: the box copy fills
// cells outside the level with zeros; each halo strip rebuilds its
// out-of-level cells as the odd reflection of in-level cells of the same
// staged plane (Eq. error_ghost, repeated: the mirror of cell -1-k is -cell k).
struct FixDesc {
    int dst;        // strip offset in the plane; -1: this thread owns no strip
    int srow;       // offset of the mirrored row in the plane (-1: outside the tile)
    int cols;       // mirrored local column of each cell, 8 bits each
    int masks;      // bits 0-3: cell outside the level; 4-7: mirror inside the tile; 8-11: negated
};

template <int Q, int HO, int W, int H>
__device__ __forceinline__ FixDesc make_fix(int k, int X0, int Yt, const LevelGeom& g) {
    FixDesc d;
    d.dst = -1;
    d.srow = -1;
    d.cols = 0;
    d.masks = 0;
    const int r = k / Q, q = k % Q;
    const int gy = Yt + r;
    int sy;
    const int yy = map_axis(gy, g.ny, false, &sy);
    const int rr = yy - Yt;
    const bool row_in = rr >= 0 && rr < H;
    const bool y_out = gy < 0 || gy >= g.ny;
    int masks = 0, cols = 0;
    for (int e = 0; e < 4; ++e) {
        const int gx = X0 + 4 * q + e;
        int sx;
        const int xx = map_axis(gx, g.nx, false, &sx);
        const int cc = xx - X0;
        if (y_out || gx < 0 || gx >= g.nx) {
            masks |= 1 << e;
            if (row_in && cc >= 0 && cc < W) {
                masks |= 16 << e;
                cols |= cc << (8 * e);
            }
            if (sx * sy < 0) masks |= 256 << e;
        }
    }
    d.dst = (r & 1) * HO + (r >> 1) * W + 4 * q;
    if (masks) {
        d.srow = row_in ? (rr & 1) * HO + (rr >> 1) * W : -1;
        d.cols = cols;
        d.masks = masks;
    }
    return d;
}

// The cells of one strip after a plane has landed: out-of-level cells from
// their mirrors, every cell negated when the plane is the z reflection.
__device__ __forceinline__ float4 fixed_strip(const FixDesc& d, const float* plane, float4 own, int zsign) {
    float v[4] = {own.x, own.y, own.z, own.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (d.masks & (1 << e)) {
            float m = 0.f;
            if (d.masks & (16 << e)) m = plane[d.srow + ((d.cols >> (8 * e)) & 255)];
            v[e] = (d.masks & (256 << e)) ? -m : m;
        }
        if (zsign < 0) v[e] = -v[e];
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

constexpr int kPrefetch = 8;      // TMA path: planes between the box prefetch into L2 and the first use

// Packed FP32 pairs (Blackwell f32x2 instructions): each call is two
// independent FP32 operations with the rounding of the scalar ones.
__device__ __forceinline__ unsigned long long pk(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// One strip of stage j >= 2: Y_j = ax sx + ay sy + az sz + b c + W_j.
__device__ __forceinline__ float4 later_strip(float4 c, float4 n, float4 s, float4 d, float4 u, float l, float r,
                                              float2 ax, float2 ay, float2 az, float2 bb, float4 w) {
    const float2 sx01 = make_float2(l + c.y, c.x + c.z), sx23 = make_float2(c.y + c.w, c.z + r);
    const float2 v01 = fma2(ax, sx01, fma2(ay, add2(lo2(n), lo2(s)), fma2(az, add2(lo2(d), lo2(u)), fma2(bb, lo2(c), lo2(w)))));
    const float2 v23 = fma2(ax, sx23, fma2(ay, add2(hi2(n), hi2(s)), fma2(az, add2(hi2(d), hi2(u)), fma2(bb, hi2(c), hi2(w)))));
    return cat4(v01, v23);
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}

// One strip of stage 1: Lf = L Y0 - f, Y1 = c + mu~_1 tau Lf and the combined
// fields W_2 (and W_3 for s = 3), in packed FP32 pairs (cells 0, 1 and 2, 3 of
// the strip): a thread runs two strips of a row pair, so four independent
// pairs hide the latency of the chain Lf -> Y1 -> W_j.
template <int S>
__device__ __forceinline__ void first_strip(const LeanCoef& k, float4 c, float4 n, float4 s, float4 d, float4 u,
                                            float l, float r, float4 f, float4& y1, float4& w2, float4& w3) {
    const float2 ihx = dup2(k.ihx2), ihy = dup2(k.ihy2), ihz = dup2(k.ihz2), m2s = dup2(k.m2s);
    const float2 m1t = dup2(k.m1t), k2y0 = dup2(k.k2y0), k2z = dup2(k.k2z), k2f = dup2(k.k2f);
    const float2 sx01 = make_float2(l + c.y, c.x + c.z), sx23 = make_float2(c.y + c.w, c.z + r);
    const float2 lf01 = sub2(fma2(ihx, sx01, fma2(ihy, add2(lo2(n), lo2(s)), fma2(ihz, add2(lo2(d), lo2(u)),
                                                                                    mul2(m2s, lo2(c))))), lo2(f));
    const float2 lf23 = sub2(fma2(ihx, sx23, fma2(ihy, add2(hi2(n), hi2(s)), fma2(ihz, add2(hi2(d), hi2(u)),
                                                                                    mul2(m2s, hi2(c))))), hi2(f));
    y1 = cat4(fma2(m1t, lf01, lo2(c)), fma2(m1t, lf23, hi2(c)));
    w2 = cat4(fma2(k2y0, lo2(c), fma2(k2z, lf01, mul2(k2f, lo2(f)))),
              fma2(k2y0, hi2(c), fma2(k2z, lf23, mul2(k2f, hi2(f)))));
    if (S == 3) {
        const float2 k3c = dup2(k.k3c), k3l = dup2(k.k3l), k3f = dup2(k.k3f);
        w3 = cat4(fma2(k3c, lo2(c), fma2(k3l, lf01, mul2(k3f, lo2(f)))),
                  fma2(k3c, hi2(c), fma2(k3l, lf23, mul2(k3f, hi2(f)))));
    } else {
        w3 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ float4 scale4(float k, float4 v) { return make_float4(k * v.x, k * v.y, k * v.z, k * v.w); }

__device__ __forceinline__ void store_out(float* dst, float4 v, bool vec, int n) {
    if (vec) {
        st4(dst, v);
    } else {
        dst[0] = v.x;
        if (n > 1) dst[1] = v.y;
        if (n > 2) dst[2] = v.z;
        if (n > 3) dst[3] = v.w;
    }
}

// Tensor maps of the TMA path: Y0 and f as [nz][ny/2][nx] views of their even
// (index 0) and odd (index 1) rows (row stride 2 nx), so that one box copy
// fills the even-row half or the odd-row half of a staged plane.
struct LeanMaps {
    CUtensorMap y0[2];
    CUtensorMap f[2];
};

template <int S, int ORDER, bool ZERO, int TY, bool TMA>
__global__ void __launch_bounds__(Lean<S, ZERO, TY>::NT, Lean<S, ZERO, TY>::CTAS)
k_superstep_lean(const __grid_constant__ LevelGeom g, const __grid_constant__ LeanCoef k,
                 const __grid_constant__ LeanMaps maps, const float* __restrict__ y0g,
                 const float* __restrict__ fg, float* __restrict__ outg, int tiles_x, int kchunk, int vec_ok) {
    using C = Lean<S, ZERO, TY>;
    constexpr int W = C::W, P = C::P, Q = C::Q, HQ = C::HQ, NS = C::NS;
    extern __shared__ __align__(128) float sm[];
    const int tid = threadIdx.x, lane = tid & 31;
    const int nx = g.nx, ny = g.ny, nz = g.nz, plane = nx * ny;
    const bool pz = g.per[2] != 0;
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sm + C::NFLOATS);
    const bool producer = TMA && tid == C::NT - 1;      // issues every box copy of the CTA
    if (TMA) {
        // box copies land on 128-byte boundaries: refuse a misaligned window
        if ((smem_addr(sm) & 127u) != 0) {
            if (tid == 0) {
                atomicAdd(&g_lean_wait_timeouts, 1u);
                outg[0] = __int_as_float(0x7fc00000);
            }
            return;
        }
        if (producer) {
            for (int b = 0; b < C::NBAR; ++b) mbar_init(mbar + b, 1);
            mbar_init_fence();
        }
        __syncthreads();
    }

    // ---- one segment of the stream: tile (bx, by), planes [kz0, kz1)
    auto segment = [&](int bx, int by, int kz0, int kz1) {
    const int X0 = bx * C::TX - C::HX;                  // global x of local column 0
    const int Yt = by * C::TY - NS;                     // global y of local row 0

    // ---- this thread's pipeline stage and row pair (fixed for the whole
    // stream; J = 0: loads only)
    int J, item;
    if (tid < C::T2) { J = 1; item = tid; }
    else if (NS >= 2 && tid < C::T3) { J = 2; item = tid - C::T2; }
    else if (NS == 3 && tid < C::TS) { J = 3; item = tid - C::T3; }
    else { J = 0; item = 0; }
    const int Jr = J > 0 ? J : 1;
    const int nqj = Jr == 1 ? C::nq(1) : (Jr == 2 ? C::nq(2) : C::nq(3));
    const int qloj = Jr == 1 ? C::qlo(1) : (Jr == 2 ? C::qlo(2) : C::qlo(3));
    const int nitems = J == 1 ? C::items(1) : (J == 2 ? C::items(2) : (J == 3 ? C::items(3) : 0));
    const bool active = item < nitems;
    const int it = active ? item : 0;
    const int row = Jr + 2 * (it / nqj), q = qloj + it % nqj;   // rows row, row + 1
    const int o = C::rowoff(row) + 4 * q;               // row `row` of the strip
    const int d1 = C::rowoff(row + 1) + 4 * q - o;      // row + 1 relative to o; row - 1 is d1 - W, row + 2 is W
    const bool fix_l = (it % nqj == 0) || lane == 0;
    const bool fix_r = (it % nqj == nqj - 1) || lane == 31 || !active;
    const int L = 2 * J - 1;                            // lag: stage J works on plane t - L
    // stencil stages (every pipeline stage with Y0 = 0, J >= 2 otherwise):
    // coefficients, input ring, combined-field ring, output ring
    float2 ax = dup2(0.f), ay = ax, az = ax, bb = ax;
    float kw = 0.f;
    const float* in_b = sm + o;
    const float* w_b = sm + o;
    float* out_b = sm + o;
    int w_mask = 3;
    if (ZERO && J == 1) {
        // RKL stage 2 from f: Y1 = kz[1] f folded into the coefficients, no W
        ax = dup2(k.zx);
        ay = dup2(k.zy);
        az = dup2(k.zz);
        bb = dup2(k.zb);
        in_b = sm + C::OF + o;
        out_b = sm + C::OY + o;
    } else if (ZERO && J == 2) {
        // RKL stage 3 from Y2: W_3 = kz[3] f
        ax = dup2(k.ax[3]);
        ay = dup2(k.ay[3]);
        az = dup2(k.az[3]);
        bb = dup2(k.b[3]);
        kw = k.kz[3];
        in_b = sm + C::OY + o;
        w_b = sm + C::OF + o;
        w_mask = C::RF - 1;
    } else if (J >= 2) {
        ax = dup2(J == 2 ? k.ax[2] : k.ax[3]);
        ay = dup2(J == 2 ? k.ay[2] : k.ay[3]);
        az = dup2(J == 2 ? k.az[2] : k.az[3]);
        bb = dup2(J == 2 ? k.b[2] : k.b[3]);
        in_b = sm + C::OY + (J - 2) * C::RY * P + o;
        out_b = sm + C::OY + (J - 1) * C::RY * P + o;
        if (J == 2) {
            w_b = sm + C::OW2 + o;
            w_mask = C::RW2 - 1;
        } else {
            w_b = sm + C::OW3 + o;
            w_mask = (C::RW3 > 0 ? C::RW3 : 1) - 1;
        }
    }
    // output cells of the last stage (rows row, row + 1)
    int st0 = -1, st1 = -1, st_n = 0;
    bool st_vec = false;
    if (J == NS && active) {
        const int gy = Yt + row, gx0 = X0 + 4 * q;
        if (gx0 < nx) {
            if (gy < ny) st0 = gy * nx + gx0;
            if (gy + 1 < ny) st1 = (gy + 1) * nx + gx0;
            st_n = min(4, nx - gx0);
            st_vec = vec_ok && st_n == 4;
        }
    }
    // staged-plane loads.  cp.async path: thread k < HQ stages strip k of Y0 and
    // of f.  TMA path: the producer copies two boxes per field (even rows, odd
    // rows); threads k < HQ of tiles that reach past a wall rebuild the
    // out-of-level cells of strip k.
    LoadDesc ld;
    ld.dst = -1;
    FixDesc fx;
    fx.dst = -1;
    fx.masks = 0;
    const bool wall = X0 < 0 || X0 + W > nx || Yt < 0 || Yt + C::H > ny;
    if (TMA) {
        if (tid < HQ) fx = make_fix<Q, C::HO, W, C::H>(tid, X0, Yt, g);
    } else {
        if (tid < HQ) ld = make_desc(tid, X0, Yt, g, vec_ok != 0, Q, C::HO, W);
    }
    // box coordinates: local even rows are the global rows of Yt's parity
    const int ypar = Yt & 1;
    const int ybox_e = (Yt - ypar) / 2, ybox_o = (Yt + ypar) / 2;
    const int t_first = kz0 - NS + 2;                   // stage 1 computes plane t - 1
    const int nph = (kz1 - kz0) + 3 * NS - 3;           // phases
    const int nload = kz1 + NS - t_first;               // planes t_first + v, v < nload, are staged
    const int u_store0 = kz0 - t_first + 2 * NS - 1;    // phases whose last-stage plane lies in [kz0, kz1)
    const int u_store1 = kz1 - t_first + 2 * NS - 1;
    // plane t_first + v of a ring with R slots sits in slot (v & (R - 1)); on the
    // TMA path its copies complete on mbarrier (v + 2) & 3, phase ((v + 2) >> 2) & 1
    auto stage_plane = [&](int v, int* zsign) {
        const int zz = map_axis(t_first + v, nz, pz, zsign);
        if constexpr (TMA) {
            if (producer) {
                unsigned long long* bar = mbar + ((v + 2) & 3);
                fence_proxy_async();
                mbar_expect_tx(bar, (ZERO ? 1u : 2u) * unsigned(C::H * W * sizeof(float)));
                if constexpr (!ZERO) {
                    float* d = sm + C::OY0 + (v & 3) * P;
                    tma_load(d, &maps.y0[ypar], X0, ybox_e, zz, bar);
                    tma_load(d + C::HO, &maps.y0[ypar ^ 1], X0, ybox_o, zz, bar);
                }
                float* d = sm + C::OF + (v & (C::RF - 1)) * P;
                tma_load(d, &maps.f[ypar], X0, ybox_e, zz, bar);
                tma_load(d + C::HO, &maps.f[ypar ^ 1], X0, ybox_o, zz, bar);
            }
        } else {
            const int src = zz * plane;
            if constexpr (!ZERO) issue(ld, sm + C::OY0 + (v & 3) * P, y0g + src);
            issue(ld, sm + C::OF + (v & (C::RF - 1)) * P, fg + src);
        }
    };
    // TMA path: whole boxes into L2 kPrefetch planes ahead (the per-strip copies
    // run without: a per-thread L2 prefetch there measured slower, 138.9
    // against 132.8 us per general 256^3 launch)
    auto prefetch_plane = [&](int v) {
        int zsg;
        const int zz = map_axis(t_first + v, nz, pz, &zsg);
        if constexpr (TMA) {
            if (producer) {
                if constexpr (!ZERO) {
                    tma_prefetch(&maps.y0[ypar], X0, ybox_e, zz);
                    tma_prefetch(&maps.y0[ypar ^ 1], X0, ybox_o, zz);
                }
                tma_prefetch(&maps.f[ypar], X0, ybox_e, zz);
                tma_prefetch(&maps.f[ypar ^ 1], X0, ybox_o, zz);
            }
        }
    };
    // cp.async path: the thread's own copies have landed; negate reflected cells
    auto fix_plane = [&](int v, int zsign) {
        if constexpr (!ZERO) fixup(ld, sm + C::OY0 + (v & 3) * P, zsign);
        fixup(ld, sm + C::OF + (v & (C::RF - 1)) * P, zsign);
    };
    // TMA path: wait (bounded) for plane v, then rebuild its out-of-level cells
    // (wall tiles) and negate it (z reflection).  Every thread takes the same
    // branches, so the barrier between the reads and the writes of a negated
    // plane is reached by all.  Returns false if the wait gave up.
    auto land_plane = [&](int v, int zsign) -> bool {
        const bool ok = mbar_wait(mbar + ((v + 2) & 3), ((v + 2) >> 2) & 1);
        float* pfp = sm + C::OF + (v & (C::RF - 1)) * P;
        float* pyp = sm + C::OY0 + (v & 3) * P;
        if (zsign < 0) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (ok && fx.dst >= 0) {
                a = fixed_strip(fx, pfp, ld4(pfp + fx.dst), -1);
                if constexpr (!ZERO) b = fixed_strip(fx, pyp, ld4(pyp + fx.dst), -1);
            }
            __syncthreads();
            if (ok && fx.dst >= 0) {
                st4(pfp + fx.dst, a);
                if constexpr (!ZERO) st4(pyp + fx.dst, b);
            }
        } else if (ok && wall && fx.masks) {
            st4(pfp + fx.dst, fixed_strip(fx, pfp, ld4(pfp + fx.dst), 1));
            if constexpr (!ZERO) st4(pyp + fx.dst, fixed_strip(fx, pyp, ld4(pyp + fx.dst), 1));
        }
        return ok;
    };
    // a bounded wait gave up: count it, poison the output so that the solve
    // reports a non-finite residual, and leave (every thread of the CTA agrees)
    auto give_up = [&]() {
        if (tid == 0) {
            atomicAdd(&g_lean_wait_timeouts, 1u);
            outg[0] = __int_as_float(0x7fc00000);
        }
    };

    // ---- prologue: planes t_first - 2 .. t_first; t_first + 1 stays in flight
    int zs0, zs1, zs2, zs_next = 1;
    stage_plane(-2, &zs0);
    stage_plane(-1, &zs1);
    stage_plane(0, &zs2);
    if constexpr (TMA) {
        if (1 < nload) stage_plane(1, &zs_next);
        bool ok = land_plane(-2, zs0);
        ok = land_plane(-1, zs1) && ok;
        ok = land_plane(0, zs2) && ok;
        for (int v = 2; v < kPrefetch && v < nload; ++v) prefetch_plane(v);
        if (__syncthreads_or(!ok)) {
            give_up();
            return;
        }
    } else {
        cpa_commit();
        cpa_wait_all();
        fix_plane(-2, zs0);
        fix_plane(-1, zs1);
        fix_plane(0, zs2);
        if (1 < nload) stage_plane(1, &zs_next);
        cpa_commit();
        __syncthreads();
    }

    // z window of the thread's two strips: planes p - 1 (dn) and p (cen)
    float4 dn0 = make_float4(0.f, 0.f, 0.f, 0.f), cen0 = dn0, dn1 = dn0, cen1 = dn0;
    if (J == 1) {            // stage 1 reads the staged planes -2 and -1 (Y0, or f when Y0 = 0)
        const float* base = ZERO ? sm + C::OF + o : sm + C::OY0 + o;
        const int mask = ZERO ? C::RF - 1 : 3;
        dn0 = ld4(base + (-2 & mask) * P);
        dn1 = ld4(base + (-2 & mask) * P + d1);
        cen0 = ld4(base + (-1 & mask) * P);
        cen1 = ld4(base + (-1 & mask) * P + d1);
    }

    // One phase.  (dn, cen) hold the thread's strips of planes p - 1 and p of its
    // input stage; the strips of plane p + 1 are loaded into `nxt`.  The loop
    // below rotates the three register sets by renaming (unrolled by three).
    auto phase = [&](int u, float4& dn0, float4& cen0, float4& nxt0, float4& dn1, float4& cen1, float4& nxt1) -> bool {
        const int zs_cur = zs_next;

        if (!ZERO && J == 1) {
            // ---- stage 1 on plane t - 1
            const int sp = (u - 1) & 3;
            const float* yc = sm + C::OY0 + sp * P + o;
            const float* yu = sm + C::OY0 + (u & 3) * P + o;
            const float* fp = sm + C::OF + ((u - 1) & 3) * P + o;
            nxt0 = ld4(yu);
            nxt1 = ld4(yu + d1);
            const float4 up0 = nxt0, up1 = nxt1;
            const float4 nn = ld4(yc + d1 - W), ss = ld4(yc + W);
            const float4 f0 = ld4(fp), f1 = ld4(fp + d1);
            float l0 = __shfl_up_sync(0xffffffffu, cen0.w, 1);
            float r0 = __shfl_down_sync(0xffffffffu, cen0.x, 1);
            float l1 = __shfl_up_sync(0xffffffffu, cen1.w, 1);
            float r1 = __shfl_down_sync(0xffffffffu, cen1.x, 1);
            if (fix_l) { l0 = yc[-1]; l1 = yc[d1 - 1]; }
            if (fix_r) { r0 = yc[4]; r1 = yc[d1 + 4]; }
            float4 y1a, w2a, w3a, y1b, w2b, w3b;
            first_strip<S>(k, cen0, nn, cen1, dn0, up0, l0, r0, f0, y1a, w2a, w3a);
            first_strip<S>(k, cen1, cen0, ss, dn1, up1, l1, r1, f1, y1b, w2b, w3b);
            if (active) {
                float* y1p = sm + C::OY + sp * P + o;
                float* w2p = sm + C::OW2 + sp * P + o;
                st4(y1p, y1a);
                st4(y1p + d1, y1b);
                st4(w2p, w2a);
                st4(w2p + d1, w2b);
                if (S == 3) {
                    float* w3p = sm + C::OW3 + ((u - 1) & 7) * P + o;
                    st4(w3p, w3a);
                    st4(w3p + d1, w3b);
                }
            }
        } else if (J >= 1) {
            // ---- stencil stage J on plane p = t - L
            const int in_mask = (ZERO && J == 1) ? C::RF - 1 : 3;
            const float* yc = in_b + ((u - L) & in_mask) * P;
            const float* yu = in_b + ((u - L + 1) & in_mask) * P;
            nxt0 = ld4(yu);
            nxt1 = ld4(yu + d1);
            const float4 up0 = nxt0, up1 = nxt1;
            const float4 nn = ld4(yc + d1 - W), ss = ld4(yc + W);
            float l0 = __shfl_up_sync(0xffffffffu, cen0.w, 1);
            float r0 = __shfl_down_sync(0xffffffffu, cen0.x, 1);
            float l1 = __shfl_up_sync(0xffffffffu, cen1.w, 1);
            float r1 = __shfl_down_sync(0xffffffffu, cen1.x, 1);
            if (fix_l) { l0 = yc[-1]; l1 = yc[d1 - 1]; }
            if (fix_r) { r0 = yc[4]; r1 = yc[d1 + 4]; }
            float4 wa = make_float4(0.f, 0.f, 0.f, 0.f), wb = wa;
            if (!ZERO || J >= 2) {
                const float* wp = w_b + ((u - L) & w_mask) * P;
                wa = ld4(wp);
                wb = ld4(wp + d1);
                if (ZERO) {
                    wa = scale4(kw, wa);
                    wb = scale4(kw, wb);
                }
            }
            const float4 va = later_strip(cen0, nn, cen1, dn0, up0, l0, r0, ax, ay, az, bb, wa);
            const float4 vb = later_strip(cen1, cen0, ss, dn1, up1, l1, r1, ax, ay, az, bb, wb);
            if (J < NS) {
                if (active) {
                    const int op = ((u - L) & 3) * P;
                    st4(out_b + op, va);
                    st4(out_b + op + d1, vb);
                }
            } else if (u >= u_store0 && u < u_store1) {
                float* ob = outg + (t_first + u - L) * plane;
                if (st0 >= 0) store_out(ob + st0, va, st_vec, st_n);
                if (st1 >= 0) store_out(ob + st1, vb, st_vec, st_n);
            }
        }

        // stage plane t + 2 into shared memory (its slot held plane t - 2, read
        // for the last time in the previous phase), after this phase's reads
        // (TMA path: and prefetch plane t + kPrefetch into L2)
        if (u + 2 < nload) stage_plane(u + 2, &zs_next);
        if constexpr (!TMA) cpa_commit();
        if (TMA && u + kPrefetch < nload) prefetch_plane(u + kPrefetch);

        // plane t + 1 (staged in the previous phase) has landed: fix its reflected cells
        if constexpr (TMA) {
            bool ok = true;
            if (u + 1 < nload) ok = land_plane(u + 1, zs_cur);
            return !__syncthreads_or(!ok);
        } else {
            cpa_wait_prev();
            if (u + 1 < nload) fix_plane(u + 1, zs_cur);
            __syncthreads();
            return true;
        }
    };

    float4 nx0 = make_float4(0.f, 0.f, 0.f, 0.f), nx1 = nx0;
    bool ok = true;                                 // false: a bounded wait gave up (the whole CTA agrees)
    for (int u = 0; u < nph; u += 3) {              // nph is uniform: every thread takes the same exits
        ok = phase(u, dn0, cen0, nx0, dn1, cen1, nx1);
        if (!ok || u + 1 >= nph) break;
        ok = phase(u + 1, cen0, nx0, dn0, cen1, nx1, dn1);
        if (!ok || u + 2 >= nph) break;
        ok = phase(u + 2, nx0, dn0, cen0, nx1, dn1, cen1);
        if (!ok) break;
    }
    if (!ok) give_up();
    };

    // CTA b streams planes [c kchunk, (c + 1) kchunk) of one tile: all tiles
    // share the chunk boundaries, so neighbouring tiles stream the same planes
    // at about the same time and their halo rows are served from L2
    const int cpt = (nz + kchunk - 1) / kchunk;
    const int tile = blockIdx.x / cpt, c = blockIdx.x % cpt;
    segment(tile % tiles_x, tile / tiles_x, c * kchunk, min(nz, (c + 1) * kchunk));
}

int g_lean_sms = 152;

template <int S, int ORDER, bool ZERO, int TY>
struct LeanResident {
    static int per_sm;
};
template <int S, int ORDER, bool ZERO, int TY>
int LeanResident<S, ORDER, ZERO, TY>::per_sm = 1;

LeanCoef make_lean_coef(const LevelGeom& g, int order, int s, const FusedCoef& cf) {
    LeanCoef k{};
    const double hx = g.ihx2f, hy = g.ihy2f, hz = g.ihz2f;
    const double tau = cf.tau;
    for (int j = 2; j <= s; ++j) {
        const double mt = cf.mut_tau[j];
        k.ax[j] = float(mt * hx);
        k.ay[j] = float(mt * hy);
        k.az[j] = float(mt * hz);
        k.b[j] = float(double(cf.mu[j]) - 2.0 * mt * (hx + hy + hz));
    }
    k.ihx2 = g.ihx2f;
    k.ihy2 = g.ihy2f;
    k.ihz2 = g.ihz2f;
    k.m2s = float(-2.0 * (hx + hy + hz));
    k.m1t = float(double(cf.mut1) * tau);
    const double c0_2 = order == 2 ? cf.c0[2] : 0.0, gt_2 = order == 2 ? cf.gt[2] : 0.0;
    k.k2y0 = float(double(cf.nu[2]) + c0_2);
    k.k2z = float(gt_2 * tau);
    k.k2f = float(-double(cf.mut_tau[2]));
    if (s >= 3) {
        const double c0_3 = order == 2 ? cf.c0[3] : 0.0, gt_3 = order == 2 ? cf.gt[3] : 0.0;
        const double nu3 = cf.nu[3];
        k.k3c = float(nu3 + c0_3);
        k.k3l = float(nu3 * double(cf.mut1) * tau + gt_3 * tau);
        k.k3f = float(-double(cf.mut_tau[3]));
    }
    // Y0 = 0: Z0 = -tau f, Y1 = -mu~_1 tau f
    const double y1 = -double(cf.mut1) * tau;
    k.kz[1] = float(y1);
    const double kz2 = -gt_2 * tau - double(cf.mut_tau[2]);
    k.kz[2] = float(kz2);
    // Y2 = mu~_2 tau (hx sx + hy sy + hz sz) Y1 + b_2 Y1 + kz2 f with Y1 = y1 f
    {
        const double mt = cf.mut_tau[2];
        k.zx = float(mt * hx * y1);
        k.zy = float(mt * hy * y1);
        k.zz = float(mt * hz * y1);
        k.zb = float((double(cf.mu[2]) - 2.0 * mt * (hx + hy + hz)) * y1 + kz2);
    }
    if (s >= 3) {
        const double gt_3 = order == 2 ? cf.gt[3] : 0.0;
        k.kz[3] = float(double(cf.nu[3]) * y1 - gt_3 * tau - double(cf.mut_tau[3]));
    }
    return k;
}

// A launch plan: every tile cut into equal z chunks (at least 4s planes; a
// chunk costs 3s - 3 extra pipeline phases), one resident wave of CTAs.
struct LeanPlan {
    long long tiles_x = 0, ncta = 0;
    int kchunk = 0;
    double cost = 0;     // the longest SM: CTAs per SM x phases x strip items per phase
};

template <int S, int ORDER, bool ZERO, int TY>
LeanPlan lean_plan(const LevelGeom& g) {
    using C = Lean<S, ZERO, TY>;
    LeanPlan p;
    const long long gx = (g.nx + C::TX - 1) / C::TX, gy = (g.ny + C::TY - 1) / C::TY;
    const long long slots = (long long)g_lean_sms * LeanResident<S, ORDER, ZERO, TY>::per_sm;
    long long chunks = std::max(1LL, slots / (gx * gy));
    chunks = std::min<long long>(chunks, std::max(1, g.nz / (4 * C::NS)));
    p.tiles_x = gx;
    p.kchunk = (int)((g.nz + chunks - 1) / chunks);
    p.ncta = gx * gy * ((g.nz + p.kchunk - 1) / p.kchunk);
    const long long per_sm = (p.ncta + g_lean_sms - 1) / g_lean_sms;
    const int items = C::items(1) + C::items(2) + C::items(3);
    p.cost = double(per_sm) * double(p.kchunk + 3 * C::NS - 3) * double(items);
    return p;
}

// ---- tensor maps (TMA path) --------------------------------------------------
using TensorMapEncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                          const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                          CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                          CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no link
// against the driver library); nullptr where the driver lacks it.
TensorMapEncodeTiled tensor_map_encoder() {
    static TensorMapEncodeTiled fn = []() -> TensorMapEncodeTiled {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<TensorMapEncodeTiled>(p);
    }();
    return fn;
}

// [nz][ny/2][nx] view of the rows of parity `par` of a level array: row stride
// 2 nx, box of w x h rows x 1 plane, zeros outside the level.
bool encode_rows(CUtensorMap* m, const float* base, int par, const LevelGeom& g, int w, int h) {
    TensorMapEncodeTiled enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {cuuint64_t(g.nx), cuuint64_t(g.ny / 2), cuuint64_t(g.nz)};
    const cuuint64_t strides[2] = {cuuint64_t(g.nx) * 2 * sizeof(float), cuuint64_t(g.nx) * g.ny * sizeof(float)};
    const cuuint32_t box[3] = {cuuint32_t(w), cuuint32_t(h), 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base + par * g.nx), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S, int ORDER, bool ZERO, int TY, bool TMA>
cudaError_t lean_launch(const LeanPlan& p, const LevelGeom& g, const LeanCoef& k, const LeanMaps& maps,
                        const float* y0, const float* f, float* out, int vec_ok, cudaStream_t st) {
    using C = Lean<S, ZERO, TY>;
    k_superstep_lean<S, ORDER, ZERO, TY, TMA><<<(unsigned)p.ncta, C::NT, C::BYTES, st>>>(g, k, maps, y0, f, out,
                                                                                          (int)p.tiles_x, p.kchunk,
                                                                                          vec_ok);
    return cudaGetLastError();
}

// The TMA path stages planes by box copies; it needs x and y walls without
// wrap-around (a box cannot wrap a periodic axis), 16-byte aligned rows
// (nx % 4 == 0, aligned arrays: the odd-row view starts nx floats in) and an
// even ny.  Other levels keep the per-strip cp.async path.
template <int S, int ORDER, bool ZERO, int TY>
cudaError_t lean_run(const LeanPlan& p, const LevelGeom& g, const LeanCoef& k, const float* y0, const float* f,
                     float* out, int vec_ok, cudaStream_t st, bool want_tma) {
    using C = Lean<S, ZERO, TY>;
    LeanMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    bool tma = want_tma && vec_ok && !g.per[0] && !g.per[1] && (g.ny % 2) == 0;
    if (tma) {
        for (int par = 0; par < 2 && tma; ++par) {
            tma = encode_rows(&maps.f[par], f, par, g, C::W, C::H / 2);
            if (!ZERO && tma) tma = encode_rows(&maps.y0[par], y0, par, g, C::W, C::H / 2);
        }
    }
    if (tma) return lean_launch<S, ORDER, ZERO, TY, true>(p, g, k, maps, y0, f, out, vec_ok, st);
    return lean_launch<S, ORDER, ZERO, TY, false>(p, g, k, maps, y0, f, out, vec_ok, st);
}

// Tiles 16 or 14 rows high: the shorter tile costs more halo per cell but can
// fill every CTA slot (256^3: 152 tiles x 2 chunks = 2 CTAs on each of 152
// SMs); the plan with the cheaper longest SM is launched.
template <int S, int ORDER, bool ZERO>
cudaError_t lean_one(const LevelGeom& g, const LeanCoef& k, const float* y0, const float* f, float* out,
                     cudaStream_t st, int tile_rows, bool tma) {
    const bool aligned = ((reinterpret_cast<uintptr_t>(y0) | reinterpret_cast<uintptr_t>(f) |
                           reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    const int vec_ok = ((g.nx & 3) == 0 && aligned) ? 1 : 0;
    const LeanPlan a = lean_plan<S, ORDER, ZERO, 16>(g), b = lean_plan<S, ORDER, ZERO, 14>(g);
    const bool use14 = tile_rows == 14 || (tile_rows != 16 && b.cost < a.cost);
    if (use14) return lean_run<S, ORDER, ZERO, 14>(b, g, k, y0, f, out, vec_ok, st, tma);
    return lean_run<S, ORDER, ZERO, 16>(a, g, k, y0, f, out, vec_ok, st, tma);
}

template <int S, int ORDER, bool ZERO, int TY, bool TMA>
cudaError_t lean_configure_kernel(int* per_sm) {
    using C = Lean<S, ZERO, TY>;
    auto kern = k_superstep_lean<S, ORDER, ZERO, TY, TMA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, C::NT, C::BYTES);
    if (e != cudaSuccess) return e;
    *per_sm = n > 0 ? n : 1;
    return cudaSuccess;
}

// Both load paths of a tile shape; the plan uses the smaller residency.
template <int S, int ORDER, bool ZERO, int TY>
cudaError_t lean_configure_one() {
    int a = 1, b = 1;
    cudaError_t e = lean_configure_kernel<S, ORDER, ZERO, TY, false>(&a);
    if (e != cudaSuccess) return e;
    if ((e = lean_configure_kernel<S, ORDER, ZERO, TY, true>(&b)) != cudaSuccess) return e;
    LeanResident<S, ORDER, ZERO, TY>::per_sm = std::min(a, b);
    return cudaSuccess;
}

template <int S, int ORDER, bool ZERO>
cudaError_t lean_configure_ty() {
    cudaError_t e = lean_configure_one<S, ORDER, ZERO, 16>();
    return e != cudaSuccess ? e : lean_configure_one<S, ORDER, ZERO, 14>();
}

template <int S>
cudaError_t lean_dispatch(int order, bool zero, const LevelGeom& g, const LeanCoef& k, const float* y0,
                          const float* f, float* out, cudaStream_t st, int rows, bool tma) {
    if (order == 1)
        return zero ? lean_one<S, 1, true>(g, k, y0, f, out, st, rows, tma)
                    : lean_one<S, 1, false>(g, k, y0, f, out, st, rows, tma);
    return zero ? lean_one<S, 2, true>(g, k, y0, f, out, st, rows, tma)
                : lean_one<S, 2, false>(g, k, y0, f, out, st, rows, tma);
}

}  // namespace

cudaError_t lean_configure() {
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&g_lean_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = lean_configure_ty<2, 1, false>()) != cudaSuccess) return e;
    if ((e = lean_configure_ty<2, 1, true>()) != cudaSuccess) return e;
    if ((e = lean_configure_ty<2, 2, false>()) != cudaSuccess) return e;
    if ((e = lean_configure_ty<2, 2, true>()) != cudaSuccess) return e;
    if ((e = lean_configure_ty<3, 1, false>()) != cudaSuccess) return e;
    if ((e = lean_configure_ty<3, 1, true>()) != cudaSuccess) return e;
    if ((e = lean_configure_ty<3, 2, false>()) != cudaSuccess) return e;
    return lean_configure_ty<3, 2, true>();
}

unsigned lean_wait_failures() {
    unsigned n = 0;
    if (cudaMemcpyFromSymbol(&n, g_lean_wait_timeouts, sizeof(n)) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_superstep_lean(const LevelGeom& g, int order, int s, bool zero_y0, const FusedCoef& cf,
                                  const float* y0, const float* f, float* out, cudaStream_t st, int tile_rows,
                                  bool tma) {
    const LeanCoef k = make_lean_coef(g, order, s, cf);
    if (s == 2) return lean_dispatch<2>(order, zero_y0, g, k, y0, f, out, st, tile_rows, tma);
    if (s == 3) return lean_dispatch<3>(order, zero_y0, g, k, y0, f, out, st, tile_rows, tma);
    return cudaErrorInvalidValue;
}

}  // namespace sg
