// Stencil kernels of the RKL-multigrid solver (sm_103a).
//
// All kernels read and write dense [nz][ny][nx] arrays (x fastest) and make the
// ghost values of Sec. 2.3 on the fly, so no ghost-fill pass and no padded
// copies exist.  Sweeps over a level stream along z ("2.5D"): a 32 x 8 thread
// block covers an x-y tile, every thread walks a z-chunk of its column keeping
// the z-1 / z / z+1 values in registers, so each cell of the stencil input is
// read from HBM once per sweep (x/y neighbours hit L1/L2), coalesced along x.
// These are HBM-bandwidth-bound kernels; no tensor cores are involved.
#include "sg_field_ops.cuh"
#include "sg_internal.cuh"

#include <algorithm>
#include <cstdint>
#include <type_traits>

namespace sg {

namespace {

constexpr int BX = 32;
constexpr int BY = 8;

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

// Norm arithmetic in the accumulator's own precision (FP32 accumulators must
// not go through the double-precision functions).
__device__ __forceinline__ float acc_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double acc_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float acc_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double acc_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float acc_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double acc_abs(double a) { return fabs(a); }

// x and y neighbours of cell (i, j, k) with the ghost rules (Sec. 2.3).
// FACES: the level carries Dirichlet data (finest level of an FP64 solve);
// without it the wall ghost is -centre (Eq. error_ghost).  Grids have fewer
// than 2^31 cells, so 32-bit offsets suffice.
template <bool FACES, typename T>
__device__ __forceinline__ void xy_neighbours(const T* u, const LevelGeom& g, int i, int j, int k,
                                              int idx, T c, T& xm, T& xp, T& ym, T& yp) {
    const int fx = k * g.ny + j;     // x faces are [nz][ny]
    const int fy = k * g.nx + i;     // y faces are [nz][nx]
    if (i > 0) xm = u[idx - 1];
    else if (g.per[0]) xm = u[idx + (g.nx - 1)];
    else if (FACES && g.face[0]) xm = T(2.0 * g.face[0][fx]) - c;
    else xm = -c;
    if (i < g.nx - 1) xp = u[idx + 1];
    else if (g.per[0]) xp = u[idx - (g.nx - 1)];
    else if (FACES && g.face[1]) xp = T(2.0 * g.face[1][fx]) - c;
    else xp = -c;
    const int sy = g.nx;
    if (j > 0) ym = u[idx - sy];
    else if (g.per[1]) ym = u[idx + (g.ny - 1) * sy];
    else if (FACES && g.face[2]) ym = T(2.0 * g.face[2][fy]) - c;
    else ym = -c;
    if (j < g.ny - 1) yp = u[idx + sy];
    else if (g.per[1]) yp = u[idx - (g.ny - 1) * sy];
    else if (FACES && g.face[3]) yp = T(2.0 * g.face[3][fy]) - c;
    else yp = -c;
}

template <bool FACES, typename T>
__device__ __forceinline__ T z_low(const T* u, const LevelGeom& g, int i, int j, int idx, int plane, T c) {
    if (g.per[2]) return u[idx + (g.nz - 1) * plane];
    if (FACES && g.face[4]) return T(2.0 * g.face[4][j * g.nx + i]) - c;
    return -c;
}

template <bool FACES, typename T>
__device__ __forceinline__ T z_high(const T* u, const LevelGeom& g, int i, int j, int idx, int plane, T c) {
    if (g.per[2]) return u[idx - (g.nz - 1) * plane];
    if (FACES && g.face[5]) return T(2.0 * g.face[5][j * g.nx + i]) - c;
    return -c;
}

// 16-byte vector loads (callers guarantee the alignment).
__device__ __forceinline__ float4 ld_f4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ double2 ld_d2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ float4 neg_f4(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// Eq. discrete_laplace_3D from the six neighbours.
template <typename T>
__device__ __forceinline__ T lap7(T c, T xm, T xp, T ym, T yp, T zm, T zp, T ihx2, T ihy2, T ihz2) {
    const T two_c = T(2) * c;
    return ((xm - two_c) + xp) * ihx2 + ((ym - two_c) + yp) * ihy2 + ((zm - two_c) + zp) * ihz2;
}

// Full 7-point Laplacian of one cell with ghost values on every side.
template <bool FACES, typename T>
__device__ __forceinline__ T lap_at(const T* u, const LevelGeom& g, int i, int j, int k) {
    const int plane = g.nx * g.ny;
    const int idx = k * plane + j * g.nx + i;
    const T c = u[idx];
    T xm, xp, ym, yp;
    xy_neighbours<FACES>(u, g, i, j, k, idx, c, xm, xp, ym, yp);
    const T zm = (k > 0) ? u[idx - plane] : z_low<FACES>(u, g, i, j, idx, plane, c);
    const T zp = (k < g.nz - 1) ? u[idx + plane] : z_high<FACES>(u, g, i, j, idx, plane, c);
    return lap7(c, xm, xp, ym, yp, zm, zp, ih2x<T>(g), ih2y<T>(g), ih2z<T>(g));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

// float -> double from the IEEE fields (subnormal floats, below 1.2e-38, become 0).
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned sgn = u & 0x80000000u, ex = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned hi, lo;
    if (ex == 0u) { hi = sgn; lo = 0u; }
    else if (ex == 255u) { hi = sgn | 0x7ff00000u | (m >> 3); lo = m << 29; }
    else { hi = sgn | ((ex + 896u) << 20) | (m >> 3); lo = m << 29; }
    return __hiloint2double((int)hi, (int)lo);
}

// double -> float by truncating the significand (within one FP32 ulp; values
// below 2^-126 become 0, beyond the FP32 range +-inf).
__device__ __forceinline__ float d2f_bits(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sgn = hi & 0x80000000u, ex = (hi >> 20) & 0x7ffu, mh = hi & 0xfffffu;
    if (ex <= 896u) return __uint_as_float(sgn);
    if (ex >= 1151u) return __uint_as_float(sgn | 0x7f800000u | ((ex == 2047u && (mh | lo)) ? 0x400000u : 0u));
    return __uint_as_float(sgn | ((ex - 896u) << 23) | (mh << 3) | (lo >> 29));
}

// A residual in the output precision: FP64 -> FP32 by the bit-level
// conversion (no FP64-pipe instruction), any other pair by the plain cast.
template <typename TO, typename TI>
__device__ __forceinline__ TO to_out(TI r) {
    return TO(r);
}
template <>
__device__ __forceinline__ float to_out<float, double>(double r) {
    return d2f_bits(r);
}

template <typename T>
struct CoefT {
    T tau, mut1, mu, nu, mut_tau, c0, gt;
};

int kchunk_for(const LevelGeom& g, int bx, int by);

// z-chunk with an even length (restriction and prolongation work on plane pairs).
int even_kchunk(const LevelGeom& g) {
    const int kc = kchunk_for(g, BX, BY);
    return kc + (kc & 1);
}

int kchunk_for(const LevelGeom& g, int bx, int by) {
    const long long gx = (g.nx + bx - 1) / bx, gy = (g.ny + by - 1) / by;
    const long long want = 16LL * 152;                      // 16 blocks per SM
    long long chunks = (want + gx * gy - 1) / (gx * gy);
    if (chunks < 1) chunks = 1;
    if (chunks > g.nz) chunks = g.nz;
    return (int)((g.nz + chunks - 1) / chunks);
}

// ---------------------------------------------------------------------------
// One RKL stage over a level (App. A, Eq. RKL_intermediate_source).
// ---------------------------------------------------------------------------
template <typename T, int ORDER, bool FIRST, bool FACES>
__global__ void __launch_bounds__(BX * BY)
k_stage(const LevelGeom g, const CoefT<T> cf, const T* __restrict__ ym1, const T* ym2,
        const T* y0, const T* z0, const T* __restrict__ rhs, T* out, T* z0_out, int kchunk) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int k0 = blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, g.nz);
    const int plane = g.nx * g.ny;
    int idx = k0 * plane + j * g.nx + i;
    const T ihx2 = ih2x<T>(g), ihy2 = ih2y<T>(g), ihz2 = ih2z<T>(g);
    T c = ym1[idx];
    T zm = (k0 > 0) ? ym1[idx - plane] : z_low<FACES>(ym1, g, i, j, idx, plane, c);
    for (int k = k0; k < k1; ++k, idx += plane) {
        const T zp = (k < g.nz - 1) ? ym1[idx + plane] : z_high<FACES>(ym1, g, i, j, idx, plane, c);
        T xm, xp, ym, yp;
        xy_neighbours<FACES>(ym1, g, i, j, k, idx, c, xm, xp, ym, yp);
        const T Lf = lap7(c, xm, xp, ym, yp, zm, zp, ihx2, ihy2, ihz2) - rhs[idx];
        if (FIRST) {
            const T z = cf.tau * Lf;
            out[idx] = c + cf.mut1 * z;
            if (ORDER == 2) z0_out[idx] = z;
        } else {
            T v = cf.mu * c + cf.nu * ym2[idx] + cf.mut_tau * Lf;
            if (ORDER == 2) v = v + cf.c0 * y0[idx] + cf.gt * z0[idx];
            out[idx] = v;
        }
        zm = c;
        c = zp;
    }
}

// The same stage in FP32 on strips of four x cells (homogeneous or periodic
// ghosts, nx % 4 == 0, 16-byte aligned arrays): one 16-byte load per
// neighbour row and per operand, the z neighbours carried in registers, the
// arithmetic of k_stage cell by cell.  The block is blockDim.x strips wide, so
// that levels 64 cells across fill whole warps.
template <int ORDER, bool FIRST>
__global__ void __launch_bounds__(BX * BY)
k_stage4(const LevelGeom g, const CoefT<float> cf, const float* __restrict__ ym1, const float* ym2,
         const float* y0, const float* z0, const float* __restrict__ rhs, float* out, float* z0_out, int kchunk) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;     // cells 4q .. 4q + 3
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    if (4 * q >= nx || j >= ny) return;
    const int i0 = 4 * q, plane = nx * ny;
    const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
    const float hx = g.ihx2f, hy = g.ihy2f, hz = g.ihz2f;
    const int k0 = blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, nz);
    int idx = k0 * plane + j * nx + i0;
    float4 c = ld_f4(ym1 + idx);
    float4 zm = k0 > 0 ? ld_f4(ym1 + idx - plane) : (pz ? ld_f4(ym1 + idx + (nz - 1) * plane) : neg_f4(c));
    for (int k = k0; k < k1; ++k, idx += plane) {
        const float4 zp = k < nz - 1 ? ld_f4(ym1 + idx + plane) : (pz ? ld_f4(ym1 + idx - (nz - 1) * plane) : neg_f4(c));
        const float4 ym = j > 0 ? ld_f4(ym1 + idx - nx) : (py ? ld_f4(ym1 + idx + (ny - 1) * nx) : neg_f4(c));
        const float4 yp = j < ny - 1 ? ld_f4(ym1 + idx + nx) : (py ? ld_f4(ym1 + idx - (ny - 1) * nx) : neg_f4(c));
        const float xl = i0 > 0 ? ym1[idx - 1] : (px ? ym1[idx + nx - 1] : -c.x);
        const float xr = i0 + 4 < nx ? ym1[idx + 4] : (px ? ym1[idx + 4 - nx] : -c.w);
        const float4 f = ld_f4(rhs + idx);
        float4 lf;
        lf.x = lap7(c.x, xl, c.y, ym.x, yp.x, zm.x, zp.x, hx, hy, hz) - f.x;
        lf.y = lap7(c.y, c.x, c.z, ym.y, yp.y, zm.y, zp.y, hx, hy, hz) - f.y;
        lf.z = lap7(c.z, c.y, c.w, ym.z, yp.z, zm.z, zp.z, hx, hy, hz) - f.z;
        lf.w = lap7(c.w, c.z, xr, ym.w, yp.w, zm.w, zp.w, hx, hy, hz) - f.w;
        if (FIRST) {
            const float4 z = make_float4(cf.tau * lf.x, cf.tau * lf.y, cf.tau * lf.z, cf.tau * lf.w);
            *reinterpret_cast<float4*>(out + idx) =
                make_float4(c.x + cf.mut1 * z.x, c.y + cf.mut1 * z.y, c.z + cf.mut1 * z.z, c.w + cf.mut1 * z.w);
            if (ORDER == 2) *reinterpret_cast<float4*>(z0_out + idx) = z;
        } else {
            const float4 a = ld_f4(ym2 + idx);
            float4 v = make_float4(cf.mu * c.x + cf.nu * a.x + cf.mut_tau * lf.x, cf.mu * c.y + cf.nu * a.y + cf.mut_tau * lf.y,
                                   cf.mu * c.z + cf.nu * a.z + cf.mut_tau * lf.z, cf.mu * c.w + cf.nu * a.w + cf.mut_tau * lf.w);
            if (ORDER == 2) {
                const float4 b = ld_f4(y0 + idx), d = ld_f4(z0 + idx);
                v = make_float4(v.x + cf.c0 * b.x + cf.gt * d.x, v.y + cf.c0 * b.y + cf.gt * d.y,
                                v.z + cf.c0 * b.z + cf.gt * d.z, v.w + cf.c0 * b.w + cf.gt * d.w);
            }
            *reinterpret_cast<float4*>(out + idx) = v;
        }
        zm = c;
        c = zp;
    }
}

// ---------------------------------------------------------------------------
// One colour of a red-black Gauss-Seidel / SOR sweep (Sec. 2.2.4, App. B).
// Every cell with (i + j + k) % 2 == colour solves its own row of L u = rhs,
// u <- u - omega (L u - rhs) / d, where d is the row's diagonal: -2 sum 1/h^2,
// and -1/h_d^2 more for each Dirichlet wall the cell touches (its ghost,
// -u or 2 phi_face - u, holds -u).  A cell of one colour has neighbours of the
// other colour only (periodic extents even), so the update runs in place: no
// thread reads a value another thread of the launch writes.  Each thread walks
// the cells of its colour in its column, two planes apart, carrying the plane
// between them from one cell's zp to the next cell's zm.
// ---------------------------------------------------------------------------
template <typename T, bool FACES>
__global__ void __launch_bounds__(BX * BY)
k_gsrb(const LevelGeom g, int colour, T omega, T* u, const T* __restrict__ rhs, int kchunk) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int k0 = blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, g.nz);
    const int plane = g.nx * g.ny;
    const T ihx2 = ih2x<T>(g), ihy2 = ih2y<T>(g), ihz2 = ih2z<T>(g);
    T dxy = T(-2) * (ihx2 + ihy2 + ihz2);
    if (!g.per[0]) {
        if (i == 0) dxy -= ihx2;
        if (i == g.nx - 1) dxy -= ihx2;
    }
    if (!g.per[1]) {
        if (j == 0) dxy -= ihy2;
        if (j == g.ny - 1) dxy -= ihy2;
    }
    const T inv_in = T(1) / dxy;
    int k = k0 + ((i + j + k0 + colour) & 1);
    int idx = k * plane + j * g.nx + i;
    T zm = T(0);
    bool carried = false;
    for (; k < k1; k += 2, idx += 2 * plane) {
        const T c = u[idx];
        if (!carried) zm = (k > 0) ? u[idx - plane] : z_low<FACES>(u, g, i, j, idx, plane, c);
        const T zp = (k < g.nz - 1) ? u[idx + plane] : z_high<FACES>(u, g, i, j, idx, plane, c);
        T xm, xp, ym, yp;
        xy_neighbours<FACES>(u, g, i, j, k, idx, c, xm, xp, ym, yp);
        const T r = lap7(c, xm, xp, ym, yp, zm, zp, ihx2, ihy2, ihz2) - rhs[idx];
        T inv = inv_in;
        if (!g.per[2] && (k == 0 || k == g.nz - 1)) {
            T d = dxy - ihz2;
            if (k == 0 && k == g.nz - 1) d -= ihz2;
            inv = T(1) / d;
        }
        u[idx] = c - omega * r * inv;
        zm = zp;
        carried = true;
    }
}

// ---------------------------------------------------------------------------
// The FP64 residual r = f - A phi that confirms a mixed solve (Sec. 2.1; the
// standard sign), its stencil sum in exact 64-bit fixed point.
//
// In FP64 the seven-point sum costs about seven FP64-pipe instructions per
// cell, which GB300 issues at 1/64 of the FP32 rate.  Here every operand of
// the sum (phi, and the Dirichlet ghost 2 phi_face - phi) becomes an integer
// on one scale common to the level, V = trunc(v 2^(1079 - M)), where M is the
// largest biased exponent among the phi values and, one above their own, the
// face values (a pre-pass finds it).  The conversion works on the IEEE fields
// with integer operations: |V| < 2^57, ghosts stay below 2^58 and the
// neighbour sum below 9 * 2^58, so the sum is exact in 64 bits.  Truncation
// moves an operand by less than 2^(M - 1079), 1/16 of an FP64 ulp of the
// largest operand: the integer sum is at least as close to the exact
// Laplacian as an FP64 evaluation of it.  The sum is rounded to FP64 once (to
// nearest, ties to even; integer operations again) and enters r through one
// FP64 FMA per axis, one in all when h is the same on every axis.  A level
// whose M lies outside [kFxMinExp, kFxMaxExp] (values beyond 2^-900 .. 2^900,
// or not finite) takes the FP64 stencil instead.
// ---------------------------------------------------------------------------
constexpr unsigned kFxMinExp = 1023u - 900u;
constexpr unsigned kFxMaxExp = 1023u + 900u;

// v 2^(1079 - M), truncated toward zero, for |v| < 2^(M - 1022).
__device__ __forceinline__ long long fx_from(double v, unsigned M) {
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const unsigned be = (hi >> 20) & 0x7ffu;
    const unsigned long long sig = ((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo;  // 2^52 + mantissa
    unsigned long long a;
    // v 2^(1079 - M) = sig 2^(be - M + 4); a shift of 64 or more gives 0, the
    // value of zero (and of subnormals, below 2^-1022)
    asm("shr.b64 %0, %1, %2;" : "=l"(a) : "l"(sig << 4), "r"(be ? M - be : 64u));
    const long long s = (long long)((int)hi >> 31);       // 0 or -1
    return ((long long)a ^ s) - s;
}

// x 2^(M - 1079) rounded to the nearest FP64 value (ties to even); |x| < 2^62
// and M within [kFxMinExp, kFxMaxExp] keep the result a normal number.
__device__ __forceinline__ double fx_to_f64(long long x, unsigned M) {
    if (x == 0) return 0.0;
    const unsigned long long sgn = (unsigned long long)x & 0x8000000000000000ull;
    unsigned long long a = sgn ? 0ull - (unsigned long long)x : (unsigned long long)x;
    const unsigned lz = (unsigned)__clzll((long long)a);
    a <<= lz;                                             // leading one at bit 63
    unsigned long long m = a >> 11;                       // 53 bits, leading one at bit 52
    const unsigned rest = (unsigned)a & 0x7ffu;
    m += ((rest + (unsigned)(m & 1ull)) > 0x400u) ? 1ull : 0ull;   // a carry to 2^53 moves into the exponent
    // x lies in [2^(63 - lz), 2^(64 - lz)): the value's biased exponent is
    // M + 7 - lz, and the leading one of m adds one to the field
    const unsigned long long field = (unsigned long long)(M + 6u - lz) << 52;
    return __longlong_as_double((long long)(sgn | (field + m)));
}

// ---------------------------------------------------------------------------
// Acceleration g = -grad phi by the fourth-order central difference of Sec. 3
// (Eq. 4thorder_acceleration): along each axis,
//   g_d = -(8 (phi_{+1} - phi_{-1}) - (phi_{+2} - phi_{-2})) / (12 h_d),
// the paper's -(4/3)(.)/(2h) + (1/3)(.)/(4h) over a common denominator.  Past
// a Dirichlet wall both ghost layers reflect through the face value (the
// m-th ghost is 2 phi_face - the m-th cell from the wall; zero face values
// without face data); periodic axes wrap.  FP64 throughout.
// ---------------------------------------------------------------------------
// The kernel: a 32 x 8 column tile walks its z chunk, the z neighbours in a
// five-plane register window (one load per cell), the x and y neighbours from
// the plane's tile with a two-cell halo in shared memory (double-buffered: one
// barrier per plane).  160 threads fetch the halo of each plane by the wall /
// periodic rule above; every other access is a fixed offset.
constexpr int kGravHalo = 2;
constexpr int kGravTX = BX + 2 * kGravHalo, kGravTY = BY + 2 * kGravHalo;

// The value arithmetic of the kernel, FP64 or exact fixed point (the
// confirmation residual's scale: V = trunc(phi 2^(1079 - M)), declared below):
// from() takes a stored potential, ghost() forms 2 phi_face - mirror, and
// comp() one component c (8 (a1 - b1) + (b2 - a2)).  In fixed point the
// combination is exact (|V| < 2^57, ghosts below 2^58, the combination below
// 18 * 2^58) and is rounded to FP64 once before the product with c.
struct GravF64 {
    using V = double;
    __device__ __forceinline__ V from(double v) const { return v; }
    __device__ __forceinline__ V ghost(double face, V mirror) const { return 2.0 * face - mirror; }
    __device__ __forceinline__ double comp(double c, V a1, V b1, V a2, V b2) const {
        return c * fma(8.0, a1 - b1, b2 - a2);
    }
};
struct GravFx {
    using V = long long;
    unsigned M;
    __device__ __forceinline__ V from(double v) const { return fx_from(v, M); }
    __device__ __forceinline__ V ghost(double face, V mirror) const { return fx_from(face, M - 1u) - mirror; }
    __device__ __forceinline__ double comp(double c, V a1, V b1, V a2, V b2) const {
        return c * fx_to_f64(8 * (a1 - b1) + (b2 - a2), M);
    }
};

// phi at (x, y, z) of a level with possibly out-of-range x or y (one axis at a
// time: the halo of the star stencil has no corners): the periodic image, or
// the reflection 2 phi_face - phi(mirror) past a Dirichlet wall (x, y >= 2 cells).
template <class P>
__device__ __forceinline__ typename P::V halo_phi(const double* u, const LevelGeom& g, int x, int y, int z,
                                                  const P& pv) {
    const int plane = g.nx * g.ny;
    if (x < 0 || x >= g.nx) {
        if (g.per[0]) return pv.from(u[z * plane + y * g.nx + (x < 0 ? x + g.nx : x - g.nx)]);
        const int m = x < 0 ? -1 - x : 2 * g.nx - 1 - x;
        const double* f = x < 0 ? g.face[0] : g.face[1];
        return pv.ghost(f ? f[z * g.ny + y] : 0.0, pv.from(u[z * plane + y * g.nx + m]));
    }
    if (y < 0 || y >= g.ny) {
        if (g.per[1]) return pv.from(u[z * plane + (y < 0 ? y + g.ny : y - g.ny) * g.nx + x]);
        const int m = y < 0 ? -1 - y : 2 * g.ny - 1 - y;
        const double* f = y < 0 ? g.face[2] : g.face[3];
        return pv.ghost(f ? f[z * g.nx + x] : 0.0, pv.from(u[z * plane + m * g.nx + x]));
    }
    return pv.from(u[z * plane + y * g.nx + x]);
}

// phi of column (x, y) at plane q, possibly past a z wall.
template <class P>
__device__ __forceinline__ typename P::V zcol_phi(const double* u, const LevelGeom& g, int col, int fz, int q,
                                                  const P& pv) {
    const int plane = g.nx * g.ny;
    if (q >= 0 && q < g.nz) return pv.from(u[q * plane + col]);
    if (g.per[2]) {                 // nz may be 1 (a 2D grid): wrap by the remainder
        int m = q % g.nz;
        if (m < 0) m += g.nz;
        return pv.from(u[m * plane + col]);
    }
    const int m = q < 0 ? -1 - q : 2 * g.nz - 1 - q;
    const double* f = q < 0 ? g.face[4] : g.face[5];
    return pv.ghost(f ? f[fz] : 0.0, pv.from(u[m * plane + col]));
}

template <class P>
__device__ __forceinline__ void gravity_body(const LevelGeom& g, const double* __restrict__ u,
                                             double* __restrict__ out, double cx, double cy, double cz, int kchunk,
                                             const P& pv, long long (*tile_mem)[kGravTY][kGravTX]) {
    using V = typename P::V;
    V(*tile)[kGravTY][kGravTX] = reinterpret_cast<V(*)[kGravTY][kGravTX]>(tile_mem);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < g.nx && j < g.ny;
    const int plane = g.nx * g.ny;
    const long long n = (long long)plane * g.nz;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, g.nz);
    // halo cell of this thread (tid < 160): 32 of the x halo (2 columns each
    // side, 8 rows), 128 of the y halo (2 rows each side, 32 columns)
    int hx = 0, hy = 0, sx = 0, sy = 0;
    bool halo = false;
    if (tid < 4 * BY) {
        const int r = tid % BY, c = tid / BY;                 // c: 0, 1 left; 2, 3 right
        sx = c < 2 ? c : BX + c;                              // tile columns 0, 1, BX + 2, BX + 3
        sy = r + kGravHalo;
        hx = i0 + sx - kGravHalo;
        hy = j0 + r;
        halo = hy < g.ny && (hx < g.nx + kGravHalo);
    } else if (tid < 4 * BY + 4 * BX) {
        const int t = tid - 4 * BY, c = t % BX, r = t / BX;  // r: 0, 1 below; 2, 3 above
        sx = c + kGravHalo;
        sy = r < 2 ? r : BY + r;
        hx = i0 + c;
        hy = j0 + sy - kGravHalo;
        halo = hx < g.nx && (hy < g.ny + kGravHalo);
    }
    // keep halo cells of ragged tiles inside what the stencil can reach
    if (halo) {
        const int last_x = min(g.nx, i0 + BX) - 1, last_y = min(g.ny, j0 + BY) - 1;
        if (hx > last_x + kGravHalo || hy > last_y + kGravHalo) halo = false;
    }
    const int col = active ? j * g.nx + i : 0;
    const int fz = col;
    V zm2 = V(0), zm1 = V(0), c = V(0), zp1 = V(0), zp2 = V(0);
    if (active) {
        zm2 = zcol_phi(u, g, col, fz, k0 - 2, pv);
        zm1 = zcol_phi(u, g, col, fz, k0 - 1, pv);
        c = zcol_phi(u, g, col, fz, k0, pv);
        zp1 = zcol_phi(u, g, col, fz, k0 + 1, pv);
    }
    for (int k = k0; k < k1; ++k) {
        V(*t)[kGravTX] = tile[k & 1];
        if (active) {
            zp2 = zcol_phi(u, g, col, fz, k + 2, pv);
            t[ty + kGravHalo][tx + kGravHalo] = c;
        } else if (i < g.nx + kGravHalo && j < g.ny + kGravHalo && (i < g.nx || j < g.ny)) {
            // a ragged tile: this position is the halo just past the level's last column or row
            t[ty + kGravHalo][tx + kGravHalo] = halo_phi(u, g, i, j, k, pv);
        }
        if (halo) t[sy][sx] = halo_phi(u, g, hx, hy, k, pv);
        __syncthreads();
        if (active) {
            const int a = ty + kGravHalo, b = tx + kGravHalo;
            const double gx = pv.comp(cx, t[a][b + 1], t[a][b - 1], t[a][b + 2], t[a][b - 2]);
            const double gy = pv.comp(cy, t[a + 1][b], t[a - 1][b], t[a + 2][b], t[a - 2][b]);
            const double gz = pv.comp(cz, zp1, zm1, zp2, zm2);
            const long long idx = (long long)k * plane + col;
            out[idx] = gx;
            out[n + idx] = gy;
            out[2 * n + idx] = gz;
            zm2 = zm1;
            zm1 = c;
            c = zp1;
            zp1 = zp2;
        }
    }
}

// mexp: null for FP64 arithmetic, else the fixed-point scale's pre-pass word;
// a scale out of range falls back to FP64 (the same for the whole launch).
__global__ void __launch_bounds__(BX * BY)
k_gravity_stream(const LevelGeom g, const double* __restrict__ u, double* __restrict__ out, double cx, double cy,
                 double cz, int kchunk, const unsigned* __restrict__ mexp) {
    __shared__ long long tile[2][kGravTY][kGravTX];
    const unsigned M = mexp ? *mexp : 0u;
    if (mexp && M >= kFxMinExp && M <= kFxMaxExp) gravity_body(g, u, out, cx, cy, cz, kchunk, GravFx{M}, tile);
    else gravity_body(g, u, out, cx, cy, cz, kchunk, GravF64{}, tile);
}

// ---------------------------------------------------------------------------
// Block reduction helpers (fixed order: deterministic).
// ---------------------------------------------------------------------------
// Reduction in the kernel's accumulator precision A (FP32 kernels must not
// spend FP64 issue slots on it: GB300 runs FP64 at 1/64 of the FP32 rate);
// the block's result is widened to double only when it is stored.
template <typename A>
__device__ __forceinline__ void block_reduce_write(A sumsq, A maxabs, A sum, Partial* partials, int block_id) {
    __shared__ A s_sq[32], s_mx[32], s_sum[32];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x + threadIdx.z * blockDim.x * blockDim.y;
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    for (int o = 16; o > 0; o >>= 1) {
        sumsq += __shfl_down_sync(0xffffffffu, sumsq, o);
        maxabs = acc_max(maxabs, __shfl_down_sync(0xffffffffu, maxabs, o));
        sum += __shfl_down_sync(0xffffffffu, sum, o);
    }
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) { s_sq[warp] = sumsq; s_mx[warp] = maxabs; s_sum[warp] = sum; }
    __syncthreads();
    if (warp == 0) {
        const int nw = (nthreads + 31) >> 5;
        sumsq = lane < nw ? s_sq[lane] : A(0);
        maxabs = lane < nw ? s_mx[lane] : A(0);
        sum = lane < nw ? s_sum[lane] : A(0);
        for (int o = 16; o > 0; o >>= 1) {
            sumsq += __shfl_down_sync(0xffffffffu, sumsq, o);
            maxabs = acc_max(maxabs, __shfl_down_sync(0xffffffffu, maxabs, o));
            sum += __shfl_down_sync(0xffffffffu, sum, o);
        }
        if (lane == 0) {
            Partial p;
            p.sumsq = double(sumsq); p.maxabs = double(maxabs); p.sum = double(sum); p.pad = 0.0;
            partials[block_id] = p;
        }
    }
}

// ---------------------------------------------------------------------------
// Residual r = rhs - L u (standard sign; the paper's Eq. residual is -r).
// ---------------------------------------------------------------------------
template <typename TI, typename TO, bool UNIFORM, bool FACES>
__global__ void __launch_bounds__(BX * BY)
k_residual(const LevelGeom g, const TI* __restrict__ u, const TI* __restrict__ rhs, TO* r_out,
           TI* r_full, Partial* partials, int kchunk) {
    // Norms accumulate in the output precision: an FP32 residual needs no FP64
    // arithmetic beyond the stencil itself (FP64 issue rate is the limit on GB300).
    using A = typename Acc<TO>::type;
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    A sq = A(0), mx = A(0);
    if (i < g.nx && j < g.ny) {
        const int k0 = blockIdx.z * kchunk;
        const int k1 = min(k0 + kchunk, g.nz);
        const int plane = g.nx * g.ny;
        int idx = k0 * plane + j * g.nx + i;
        const TI ihx2 = ih2x<TI>(g), ihy2 = ih2y<TI>(g), ihz2 = ih2z<TI>(g);
        const TI six = TI(-6), neg_ih2 = -ihx2;
        TI c = u[idx];
        TI zm = (k0 > 0) ? u[idx - plane] : z_low<FACES>(u, g, i, j, idx, plane, c);
        for (int k = k0; k < k1; ++k, idx += plane) {
            const TI zp = (k < g.nz - 1) ? u[idx + plane] : z_high<FACES>(u, g, i, j, idx, plane, c);
            TI xm, xp, ym, yp;
            xy_neighbours<FACES>(u, g, i, j, k, idx, c, xm, xp, ym, yp);
            TI r;
            if (UNIFORM) {
                // h equal on all axes: r = f - (sum of 6 neighbours - 6 c) / h^2,
                // 5 adds and 2 fused multiply-adds.
                const TI s6 = ((xm + xp) + (ym + yp)) + (zm + zp);
                r = fma(neg_ih2, fma(six, c, s6), rhs[idx]);
            } else {
                r = rhs[idx] - lap7(c, xm, xp, ym, yp, zm, zp, ihx2, ihy2, ihz2);
            }
            const TO ro = to_out<TO>(r);
            if (r_out) r_out[idx] = ro;
            if (r_full) r_full[idx] = r;
            const A ra = A(ro);
            sq = acc_fma(ra, ra, sq);
            mx = acc_max(mx, acc_abs(ra));
            zm = c;
            c = zp;
        }
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_reduce_write<A>(sq, mx, A(0), partials, bid);
}

// The residual of phi = 0 (f minus the face terms) for an FP32 output, in two
// launches so that no warp runs the FP64 face arithmetic for cells off the
// walls: every cell's r = f by 4-cell strips (the norm over the cells without a
// face term), then the cells next to a Dirichlet wall with face data, each
// counted once, with their face terms and their share of the norm.
__device__ __forceinline__ bool face_cell(const LevelGeom& g, int i, int j, int k) {
    return (!g.per[0] && ((i == 0 && g.face[0]) || (i == g.nx - 1 && g.face[1]))) ||
           (!g.per[1] && ((j == 0 && g.face[2]) || (j == g.ny - 1 && g.face[3]))) ||
           (!g.per[2] && ((k == 0 && g.face[4]) || (k == g.nz - 1 && g.face[5])));
}

// f minus the face terms of cell (i, j, k) (the Laplacian of zero with the
// Dirichlet ghosts 2 face - 0).
template <bool UNIFORM>
__device__ __forceinline__ double zero_face_residual(const LevelGeom& g, const double* rhs, int i, int j, int k) {
    const int idx = (k * g.ny + j) * g.nx + i;
    const bool dx = !g.per[0], dy = !g.per[1], dz = !g.per[2];
    double xm = 0.0, xp = 0.0, ym = 0.0, yp = 0.0, zm = 0.0, zp = 0.0;
    const int fx = k * g.ny + j, fy = k * g.nx + i, fz = j * g.nx + i;
    if (dx && i == 0 && g.face[0]) xm = 2.0 * g.face[0][fx];
    if (dx && i == g.nx - 1 && g.face[1]) xp = 2.0 * g.face[1][fx];
    if (dy && j == 0 && g.face[2]) ym = 2.0 * g.face[2][fy];
    if (dy && j == g.ny - 1 && g.face[3]) yp = 2.0 * g.face[3][fy];
    if (dz && k == 0 && g.face[4]) zm = 2.0 * g.face[4][fz];
    if (dz && k == g.nz - 1 && g.face[5]) zp = 2.0 * g.face[5][fz];
    if (UNIFORM) {
        const double s6 = ((xm + xp) + (ym + yp)) + (zm + zp);
        return fma(-g.ihx2, fma(-6.0, 0.0, s6), rhs[idx]);
    }
    return rhs[idx] - lap7(0.0, xm, xp, ym, yp, zm, zp, g.ihx2, g.ihy2, g.ihz2);
}

constexpr int kWallBlocks = 256;

__global__ void __launch_bounds__(BX * BY)
k_residual_zero4(const LevelGeom g, const double* __restrict__ rhs, float* __restrict__ r_out,
                 double* __restrict__ r_full, Partial* partials, int kchunk) {
    const int q = blockIdx.x * BX + threadIdx.x;        // strip: cells 4q .. 4q + 3
    const int j = blockIdx.y * BY + threadIdx.y;
    float sq = 0.0f, mx = 0.0f;
    if (4 * q < g.nx && j < g.ny) {
        const int i0 = 4 * q, plane = g.nx * g.ny;
        const int k0 = blockIdx.z * kchunk;
        const int k1 = min(k0 + kchunk, g.nz);
        int idx = k0 * plane + j * g.nx + i0;
#pragma unroll 2
        for (int k = k0; k < k1; ++k, idx += plane) {
            const double2 a = ld_d2(rhs + idx), b = ld_d2(rhs + idx + 2);
            if (r_full) {
                *reinterpret_cast<double2*>(r_full + idx) = a;
                *reinterpret_cast<double2*>(r_full + idx + 2) = b;
            }
            const float4 v = make_float4(d2f_bits(a.x), d2f_bits(a.y), d2f_bits(b.x), d2f_bits(b.y));
            if (r_out) *reinterpret_cast<float4*>(r_out + idx) = v;
            const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float x = face_cell(g, i0 + e, j, k) ? 0.0f : c[e];     // wall cells: the second pass
                sq = fmaf(x, x, sq);
                mx = fmaxf(mx, fabsf(x));
            }
        }
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_reduce_write<float>(sq, mx, 0.0f, partials, bid);
}

// The cells next to a Dirichlet wall with face data, each once: the x faces
// whole, the y faces without the x-face columns, the z faces without both.
template <bool UNIFORM>
__global__ void __launch_bounds__(BX * BY)
k_residual_zero_walls(const LevelGeom g, const double* __restrict__ rhs, float* __restrict__ r_out,
                      double* __restrict__ r_full, Partial* partials) {
    const bool dx = !g.per[0], dy = !g.per[1], dz = !g.per[2];
    const bool fx0 = dx && g.face[0], fx1 = dx && g.face[1] && g.nx > 1;
    const bool fy0 = dy && g.face[2], fy1 = dy && g.face[3] && g.ny > 1;
    const bool fz0 = dz && g.face[4], fz1 = dz && g.face[5] && g.nz > 1;
    const int ilo = fx0 ? 1 : 0, ihi = fx1 ? g.nx - 2 : g.nx - 1, nxi = max(0, ihi - ilo + 1);
    const int jlo = fy0 ? 1 : 0, jhi = fy1 ? g.ny - 2 : g.ny - 1, nyj = max(0, jhi - jlo + 1);
    const long long sx = (long long)g.ny * g.nz, sy = (long long)nxi * g.nz, sz = (long long)nxi * nyj;
    const long long seg[6] = {fx0 ? sx : 0, fx1 ? sx : 0, fy0 ? sy : 0, fy1 ? sy : 0, fz0 ? sz : 0, fz1 ? sz : 0};
    const long long total = seg[0] + seg[1] + seg[2] + seg[3] + seg[4] + seg[5];
    const int tid = threadIdx.x + threadIdx.y * BX;
    float sq = 0.0f, mx = 0.0f;
    for (long long t = (long long)blockIdx.x * (BX * BY) + tid; t < total; t += (long long)gridDim.x * (BX * BY)) {
        long long u = t;
        int s = 0;
        while (u >= seg[s]) u -= seg[s++];
        int i, j, k;
        if (s < 2) {                                     // x face: (j, k)
            i = s == 0 ? 0 : g.nx - 1;
            j = (int)(u % g.ny);
            k = (int)(u / g.ny);
        } else if (s < 4) {                              // y face: (i, k)
            j = s == 2 ? 0 : g.ny - 1;
            i = ilo + (int)(u % nxi);
            k = (int)(u / nxi);
        } else {                                         // z face: (i, j)
            k = s == 4 ? 0 : g.nz - 1;
            i = ilo + (int)(u % nxi);
            j = jlo + (int)(u / nxi);
        }
        const double r = zero_face_residual<UNIFORM>(g, rhs, i, j, k);
        const int idx = (k * g.ny + j) * g.nx + i;
        const float ro = d2f_bits(r);
        if (r_out) r_out[idx] = ro;
        if (r_full) r_full[idx] = r;
        sq = fmaf(ro, ro, sq);
        mx = fmaxf(mx, fabsf(ro));
    }
    block_reduce_write<float>(sq, mx, 0.0f, partials, blockIdx.x);
}

// The same residual for u = 0 (a solve that starts from a zero potential):
// every neighbour is zero except the ghosts of a Dirichlet wall with face data
// (2 g, Eq. solution_ghost), so r = f away from such walls.  Next to them the
// sums are formed in the order of k_residual (the same value bit for bit, up
// to the sign of an exact zero).  Whether a cell touches such a wall is
// decided per column and per end plane, outside the z loop, so cells away
// from the walls do no FP64 stencil arithmetic and u is never read.
template <typename TO, bool UNIFORM, bool FACES>
__global__ void __launch_bounds__(BX * BY)
k_residual_zero(const LevelGeom g, const double* __restrict__ rhs, TO* r_out, double* r_full, Partial* partials,
                int kchunk) {
    using A = typename Acc<TO>::type;
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    A sq = A(0), mx = A(0);
    if (i < g.nx && j < g.ny) {
        const int k0 = blockIdx.z * kchunk;
        const int k1 = min(k0 + kchunk, g.nz);
        const int plane = g.nx * g.ny;
        const bool dx = !g.per[0], dy = !g.per[1], dz = !g.per[2];
        auto emit = [&](int idx, double r) {
            const TO ro = to_out<TO>(r);
            if (r_out) r_out[idx] = ro;
            if (r_full) r_full[idx] = r;
            const A ra = A(ro);
            sq = acc_fma(ra, ra, sq);
            mx = acc_max(mx, acc_abs(ra));
        };
        // a cell next to a Dirichlet wall with face data: f minus the face terms
        auto wall_cell = [&](int k) {
            const int idx = (k * g.ny + j) * g.nx + i;
            double xm = 0.0, xp = 0.0, ym = 0.0, yp = 0.0, zm = 0.0, zp = 0.0;
            const int fx = k * g.ny + j, fy = k * g.nx + i, fz = j * g.nx + i;
            if (dx && i == 0 && g.face[0]) xm = 2.0 * g.face[0][fx];
            if (dx && i == g.nx - 1 && g.face[1]) xp = 2.0 * g.face[1][fx];
            if (dy && j == 0 && g.face[2]) ym = 2.0 * g.face[2][fy];
            if (dy && j == g.ny - 1 && g.face[3]) yp = 2.0 * g.face[3][fy];
            if (dz && k == 0 && g.face[4]) zm = 2.0 * g.face[4][fz];
            if (dz && k == g.nz - 1 && g.face[5]) zp = 2.0 * g.face[5][fz];
            double r;
            if (UNIFORM) {
                const double s6 = ((xm + xp) + (ym + yp)) + (zm + zp);
                r = fma(-g.ihx2, fma(-6.0, 0.0, s6), rhs[idx]);
            } else {
                r = rhs[idx] - lap7(0.0, xm, xp, ym, yp, zm, zp, g.ihx2, g.ihy2, g.ihz2);
            }
            emit(idx, r);
        };
        const bool wall_xy = FACES && ((dx && (i == 0 || i == g.nx - 1)) || (dy && (j == 0 || j == g.ny - 1)));
        if (wall_xy) {
            for (int k = k0; k < k1; ++k) wall_cell(k);
        } else {
            // the planes next to a z wall with face data take the face terms
            const bool zlo = FACES && dz && k0 == 0, zhi = FACES && dz && k1 == g.nz;
            const int a = zlo ? 1 : k0, b = zhi ? g.nz - 1 : k1;
            if (zlo) wall_cell(0);
            int idx = a * plane + j * g.nx + i;
            for (int k = a; k < b; ++k, idx += plane) emit(idx, rhs[idx]);
            if (zhi) wall_cell(g.nz - 1);
        }
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_reduce_write<A>(sq, mx, A(0), partials, bid);
}

// ---------------------------------------------------------------------------
// Residual fused with the 8-child restriction (Eq. restriction_example_3D).
// A 32 x 8 block streams fine planes along z (2.5D, z-neighbours in
// registers); the 2 x 2 x 2 child sum is formed by a lane shuffle (x pair),
// the register accumulator (z pair) and shared memory (y pair, neighbouring
// warps), and the coarse value (1/8 of it) is written once.  Needs even
// nx, ny, nz (true on every level that has a coarser one).
// ---------------------------------------------------------------------------
template <typename T, bool FACES>
__global__ void __launch_bounds__(BX * BY)
k_residual_restrict(const LevelGeom g, const T* __restrict__ u, const T* __restrict__ rhs, T* coarse,
                    Partial* partials, int kchunk) {
    using A = typename Acc<T>::type;
    __shared__ T s_acc[BY][BX];
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const bool active = i < g.nx && j < g.ny;
    const int cnx = g.nx >> 1, cny = g.ny >> 1;
    const int k0 = blockIdx.z * kchunk;                 // even
    const int k1 = min(k0 + kchunk, g.nz);
    const int plane = g.nx * g.ny;
    const T ihx2 = ih2x<T>(g), ihy2 = ih2y<T>(g), ihz2 = ih2z<T>(g);
    A sq = A(0), mx = A(0), csum = A(0);
    int idx = k0 * plane + (active ? j : 0) * g.nx + (active ? i : 0);
    T c = T(0), zm = T(0);
    if (active) {
        c = u[idx];
        zm = (k0 > 0) ? u[idx - plane] : z_low<FACES>(u, g, i, j, idx, plane, c);
    }
    T acc = T(0);
    for (int k = k0; k < k1; ++k, idx += plane) {
        T r = T(0);
        if (active) {
            const T zp = (k < g.nz - 1) ? u[idx + plane] : z_high<FACES>(u, g, i, j, idx, plane, c);
            T xm, xp, ym, yp;
            xy_neighbours<FACES>(u, g, i, j, k, idx, c, xm, xp, ym, yp);
            r = rhs[idx] - lap7(c, xm, xp, ym, yp, zm, zp, ihx2, ihy2, ihz2);
            const A ra = A(r);
            sq += ra * ra;
            mx = acc_max(mx, acc_abs(ra));
            zm = c;
            c = zp;
        }
        const T rx = r + __shfl_xor_sync(0xffffffffu, r, 1);      // x pair
        if ((k & 1) == 0) {
            acc = rx;                                               // first plane of the z pair
        } else {
            acc = acc + rx;                                         // second plane of the z pair
            s_acc[threadIdx.y][threadIdx.x] = acc;
            __syncthreads();
            if (((threadIdx.x | threadIdx.y) & 1) == 0 && active) {
                const T cval = (s_acc[threadIdx.y][threadIdx.x] + s_acc[threadIdx.y + 1][threadIdx.x]) * T(0.125);
                const int I = i >> 1, J = j >> 1, K = k >> 1;
                if (coarse) coarse[(K * cny + J) * cnx + I] = cval;
                csum += A(cval);
            }
            __syncthreads();
        }
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_reduce_write<A>(sq, mx, csum, partials, bid);
}

// FP32 residual + restriction on homogeneous ghosts, for nx % 4 == 0 and
// 16-byte aligned arrays: a thread owns a strip of four x cells on a pair of
// rows (2J, 2J + 1) and streams z, so each 2 x 2 x 2 block of the 8-cell mean
// (Eq. restriction_example_3D) is summed in its registers, with no shared
// memory or barrier; the z neighbours are carried in registers.
__global__ void __launch_bounds__(BX * BY, 4)
k_residual_restrict4(const LevelGeom g, const float* __restrict__ u, const float* __restrict__ rhs,
                     float* __restrict__ coarse, Partial* partials, int kchunk) {
    const int q = blockIdx.x * BX + threadIdx.x;        // cells 4q .. 4q + 3
    const int jp = blockIdx.y * BY + threadIdx.y;       // rows 2 jp, 2 jp + 1
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    float sq = 0.0f, mx = 0.0f, csum = 0.0f;
    if (4 * q < nx && 2 * jp < ny) {
        const int i0 = 4 * q, j0 = 2 * jp, plane = nx * ny;
        const int cnx = nx >> 1, cny = ny >> 1;
        const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
        const float hx = g.ihx2f, hy = g.ihy2f, hz = g.ihz2f;
        const int k0 = blockIdx.z * kchunk;             // even
        const int k1 = min(k0 + kchunk, nz);
        int idx = k0 * plane + j0 * nx + i0;
        float4 ca = ld_f4(u + idx), cb = ld_f4(u + idx + nx);
        float4 za = k0 > 0 ? ld_f4(u + idx - plane) : (pz ? ld_f4(u + idx + (nz - 1) * plane) : neg_f4(ca));
        float4 zb = k0 > 0 ? ld_f4(u + idx + nx - plane) : (pz ? ld_f4(u + idx + nx + (nz - 1) * plane) : neg_f4(cb));
        float2 acc = make_float2(0.0f, 0.0f);
        for (int k = k0; k < k1; ++k, idx += plane) {
            const bool top = k == nz - 1;
            const float4 zpa = !top ? ld_f4(u + idx + plane) : (pz ? ld_f4(u + idx - (nz - 1) * plane) : neg_f4(ca));
            const float4 zpb = !top ? ld_f4(u + idx + nx + plane) : (pz ? ld_f4(u + idx + nx - (nz - 1) * plane) : neg_f4(cb));
            const float4 ym = j0 > 0 ? ld_f4(u + idx - nx) : (py ? ld_f4(u + idx + (ny - 1) * nx) : neg_f4(ca));
            const float4 yp = j0 + 2 < ny ? ld_f4(u + idx + 2 * nx) : (py ? ld_f4(u + idx + (2 - ny) * nx) : neg_f4(cb));
            const float xla = i0 > 0 ? u[idx - 1] : (px ? u[idx + nx - 1] : -ca.x);
            const float xra = i0 + 4 < nx ? u[idx + 4] : (px ? u[idx + 4 - nx] : -ca.w);
            const float xlb = i0 > 0 ? u[idx + nx - 1] : (px ? u[idx + 2 * nx - 1] : -cb.x);
            const float xrb = i0 + 4 < nx ? u[idx + nx + 4] : (px ? u[idx + 4] : -cb.w);
            const float4 fa = ld_f4(rhs + idx), fb = ld_f4(rhs + idx + nx);
            // row a: y neighbours ym (row 2J - 1) and cb (row 2J + 1); row b: ca and yp
            const float r0 = fa.x - lap7(ca.x, xla, ca.y, ym.x, cb.x, za.x, zpa.x, hx, hy, hz);
            const float r1 = fa.y - lap7(ca.y, ca.x, ca.z, ym.y, cb.y, za.y, zpa.y, hx, hy, hz);
            const float r2 = fa.z - lap7(ca.z, ca.y, ca.w, ym.z, cb.z, za.z, zpa.z, hx, hy, hz);
            const float r3 = fa.w - lap7(ca.w, ca.z, xra, ym.w, cb.w, za.w, zpa.w, hx, hy, hz);
            const float r4 = fb.x - lap7(cb.x, xlb, cb.y, ca.x, yp.x, zb.x, zpb.x, hx, hy, hz);
            const float r5 = fb.y - lap7(cb.y, cb.x, cb.z, ca.y, yp.y, zb.y, zpb.y, hx, hy, hz);
            const float r6 = fb.z - lap7(cb.z, cb.y, cb.w, ca.z, yp.z, zb.z, zpb.z, hx, hy, hz);
            const float r7 = fb.w - lap7(cb.w, cb.z, xrb, ca.w, yp.w, zb.w, zpb.w, hx, hy, hz);
            sq = fmaf(r0, r0, fmaf(r1, r1, fmaf(r2, r2, fmaf(r3, r3, sq))));
            sq = fmaf(r4, r4, fmaf(r5, r5, fmaf(r6, r6, fmaf(r7, r7, sq))));
            mx = fmaxf(mx, fmaxf(fmaxf(fmaxf(fabsf(r0), fabsf(r1)), fmaxf(fabsf(r2), fabsf(r3))),
                                 fmaxf(fmaxf(fabsf(r4), fabsf(r5)), fmaxf(fabsf(r6), fabsf(r7)))));
            const float2 s2 = make_float2((r0 + r1) + (r4 + r5), (r2 + r3) + (r6 + r7));
            if ((k & 1) == 0) {
                acc = s2;
            } else {
                const float2 cv = make_float2((acc.x + s2.x) * 0.125f, (acc.y + s2.y) * 0.125f);
                if (coarse) *reinterpret_cast<float2*>(coarse + ((k >> 1) * cny + jp) * cnx + 2 * q) = cv;
                csum += cv.x + cv.y;
            }
            za = ca;
            ca = zpa;
            zb = cb;
            cb = zpb;
        }
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_reduce_write<float>(sq, mx, csum, partials, bid);
}

// ---------------------------------------------------------------------------
// Prolongation + correction (Eq. prolongation_example_3D): every fine cell
// takes (27 A + 9 (B + D + E) + 3 (C + F + H) + G) / 64 from its parent A and
// the parent's neighbours on the fine cell's side, and adds it to fine_u.
// The weights factor as (3, 1) per axis: a thread owns one fine (x, y)
// column, forms q(K) = sum over its 2 x 2 coarse (x, y) of (3|1)(3|1) C[K]
// once per coarse plane K, and streams z: fine plane 2K takes
// 3 q(K) + q(K-1), fine plane 2K+1 takes 3 q(K) + q(K+1), over 64.
// Coarse ghosts follow Eq. error_ghost axis by axis (index mirrored, sign
// flipped per wall) or wrap (periodic).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BX * BY)
k_prolong_correct(const LevelGeom g, const T* __restrict__ coarse, T* fine_u, int kchunk) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int cnx = g.nx >> 1, cny = g.ny >> 1, cnz = g.nz >> 1;
    const int cplane = cnx * cny;
    // coarse x / y indices of the parent (a) and the side neighbour (b), with sign
    const int Ia = i >> 1, Ja = j >> 1;
    int Ib = Ia + ((i & 1) ? 1 : -1), Jb = Ja + ((j & 1) ? 1 : -1);
    T sx = T(1), sy = T(1);
    if (Ib < 0 || Ib >= cnx) {
        if (g.per[0]) Ib = (Ib + cnx) % cnx;
        else { Ib = Ia; sx = T(-1); }
    }
    if (Jb < 0 || Jb >= cny) {
        if (g.per[1]) Jb = (Jb + cny) % cny;
        else { Jb = Ja; sy = T(-1); }
    }
    const int oaa = Ja * cnx + Ia, oab = Ja * cnx + Ib;
    const int oba = Jb * cnx + Ia, obb = Jb * cnx + Ib;
    auto q = [&](int K) -> T {                          // (x, y) interpolant of coarse plane K
        T sign = T(1);
        if (K < 0) { if (g.per[2]) K += cnz; else { K = 0; sign = T(-1); } }
        else if (K >= cnz) { if (g.per[2]) K -= cnz; else { K = cnz - 1; sign = T(-1); } }
        const T* cp = coarse + K * cplane;
        const T v = T(9) * cp[oaa] + T(3) * sx * cp[oab] + T(3) * sy * cp[oba] + sx * sy * cp[obb];
        return sign * v;
    };
    const int k0 = blockIdx.z * kchunk;                 // even
    const int k1 = min(k0 + kchunk, g.nz);
    const int plane = g.nx * g.ny;
    int idx = k0 * plane + j * g.nx + i;
    int K = k0 >> 1;
    T qm = q(K - 1), q0 = q(K), qp = q(K + 1);
    const T w = T(1.0 / 64.0);
    for (int k = k0; k < k1; k += 2, idx += 2 * plane) {
        fine_u[idx] = fine_u[idx] + (T(3) * q0 + qm) * w;
        if (k + 1 < k1) fine_u[idx + plane] = fine_u[idx + plane] + (T(3) * q0 + qp) * w;
        ++K;
        qm = q0;
        q0 = qp;
        if (k + 2 < k1) qp = q(K + 1);
    }
}

// ---- two-dimensional levels (Sec. 2.2: nz = 1, no z term) -------------------
// Residual + 4-cell restriction (Eq. restriction_example_2D): r = rhs - L u by
// the five-point operator (Eq. discrete_laplace_2D; on a 2D level the z
// neighbours are the cell itself and 1 / h_z^2 is zero, so the seven-point
// form reduces to it exactly), the coarse value the mean of a 2 x 2 block: the
// x pair by a shuffle, the y pair through shared memory.
template <typename T, bool FACES>
__global__ void __launch_bounds__(BX * BY)
k_residual_restrict2d(const LevelGeom g, const T* __restrict__ u, const T* __restrict__ rhs, T* coarse,
                      Partial* partials) {
    using A = typename Acc<T>::type;
    __shared__ T s_acc[BY][BX];
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const bool active = i < g.nx && j < g.ny;
    A sq = A(0), mx = A(0), csum = A(0);
    T r = T(0);
    if (active) {
        const int idx = j * g.nx + i;
        const T c = u[idx];
        T xm, xp, ym, yp;
        xy_neighbours<FACES>(u, g, i, j, 0, idx, c, xm, xp, ym, yp);
        const T two_c = T(2) * c;
        r = rhs[idx] - (((xm - two_c) + xp) * ih2x<T>(g) + ((ym - two_c) + yp) * ih2y<T>(g));
        const A ra = A(r);
        sq = ra * ra;
        mx = acc_abs(ra);
    }
    const T rx = r + __shfl_xor_sync(0xffffffffu, r, 1);          // x pair
    s_acc[threadIdx.y][threadIdx.x] = rx;
    __syncthreads();
    if (((threadIdx.x | threadIdx.y) & 1) == 0 && active) {
        const T cval = (s_acc[threadIdx.y][threadIdx.x] + s_acc[threadIdx.y + 1][threadIdx.x]) * T(0.25);
        if (coarse) coarse[(j >> 1) * (g.nx >> 1) + (i >> 1)] = cval;
        csum = A(cval);
    }
    block_reduce_write<A>(sq, mx, csum, partials, blockIdx.x + gridDim.x * blockIdx.y);
}

// Prolongation + correction of a 2D level (Eq. prolongation_example_2D): each
// fine cell adds (9 A + 3 B + 3 C + D) / 16, A its parent, B and C the parent's
// neighbours towards the cell along x and y, D the one between them; coarse
// ghosts follow the level's rule (-e at a Dirichlet wall, the periodic image).
template <typename T>
__global__ void __launch_bounds__(BX * BY)
k_prolong_correct2d(const LevelGeom g, const T* __restrict__ coarse, T* fine_u) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int cnx = g.nx >> 1, cny = g.ny >> 1;
    const int Ia = i >> 1, Ja = j >> 1;
    int Ib = Ia + ((i & 1) ? 1 : -1), Jb = Ja + ((j & 1) ? 1 : -1);
    T sx = T(1), sy = T(1);
    if (Ib < 0 || Ib >= cnx) {
        if (g.per[0]) Ib = (Ib + cnx) % cnx;
        else { Ib = Ia; sx = T(-1); }
    }
    if (Jb < 0 || Jb >= cny) {
        if (g.per[1]) Jb = (Jb + cny) % cny;
        else { Jb = Ja; sy = T(-1); }
    }
    const T v = T(9) * coarse[Ja * cnx + Ia] + T(3) * sx * coarse[Ja * cnx + Ib] +
                T(3) * sy * coarse[Jb * cnx + Ia] + sx * sy * coarse[Jb * cnx + Ib];
    const int idx = j * g.nx + i;
    fine_u[idx] = fine_u[idx] + v * T(1.0 / 16.0);
}

// The same prolongation + correction for FP32, nx % 4 == 0 and aligned
// arrays: a thread owns a strip of four fine x cells on a pair of fine rows
// (2J, 2J + 1).  Per coarse plane it reads coarse x = 2q - 1 .. 2q + 2 on rows
// J - 1 .. J + 1 (ghosts by the same rules), forms the x interpolants (3, 1),
// then the y interpolants of its two rows, and streams z with 16-byte
// read-modify-writes of the fine strips.
__global__ void __launch_bounds__(BX * BY)
k_prolong_correct4(const LevelGeom g, const float* __restrict__ coarse, float* __restrict__ fine_u, int kchunk) {
    const int q = blockIdx.x * BX + threadIdx.x;
    const int J = blockIdx.y * BY + threadIdx.y;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    if (4 * q >= nx || 2 * J >= ny) return;
    const int cnx = nx >> 1, cny = ny >> 1, cnz = nz >> 1, cplane = cnx * cny;
    const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
    // coarse x = 2q - 1 and 2q + 2 with their ghost rule; rows J - 1, J + 1 likewise
    int xl = 2 * q - 1, xr = 2 * q + 2;
    float sl = 1.0f, sr = 1.0f;
    if (xl < 0) { if (px) xl += cnx; else { xl = 0; sl = -1.0f; } }
    if (xr >= cnx) { if (px) xr -= cnx; else { xr = cnx - 1; sr = -1.0f; } }
    int ym = J - 1, yp = J + 1;
    float sym = 1.0f, syp = 1.0f;
    if (ym < 0) { if (py) ym += cny; else { ym = 0; sym = -1.0f; } }
    if (yp >= cny) { if (py) yp -= cny; else { yp = cny - 1; syp = -1.0f; } }
    const int rm = ym * cnx, r0 = J * cnx, rp = yp * cnx;
    // (x, y) interpolants of coarse plane K for fine rows a = 2J and b = 2J + 1
    auto interp = [&](int K, float4& qa, float4& qb) {
        float sz = 1.0f;
        if (K < 0) { if (pz) K += cnz; else { K = 0; sz = -1.0f; } }
        else if (K >= cnz) { if (pz) K -= cnz; else { K = cnz - 1; sz = -1.0f; } }
        const float* cp = coarse + K * cplane;
        float4 x[3];
        const int rows[3] = {rm, r0, rp};
        const float ys[3] = {sym, 1.0f, syp};
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const float* row = cp + rows[t];
            const float2 c2 = *reinterpret_cast<const float2*>(row + 2 * q);
            const float cl = sl * row[xl], cr = sr * row[xr];
            const float sg = ys[t] * sz;
            x[t] = make_float4(sg * (3.0f * c2.x + cl), sg * (3.0f * c2.x + c2.y), sg * (3.0f * c2.y + c2.x),
                               sg * (3.0f * c2.y + cr));
        }
        qa = make_float4(3.0f * x[1].x + x[0].x, 3.0f * x[1].y + x[0].y, 3.0f * x[1].z + x[0].z, 3.0f * x[1].w + x[0].w);
        qb = make_float4(3.0f * x[1].x + x[2].x, 3.0f * x[1].y + x[2].y, 3.0f * x[1].z + x[2].z, 3.0f * x[1].w + x[2].w);
    };
    const int k0 = blockIdx.z * kchunk;                 // even
    const int k1 = min(k0 + kchunk, nz);
    const int plane = nx * ny;
    int idx = k0 * plane + 2 * J * nx + 4 * q;
    int K = k0 >> 1;
    float4 qma, qmb, q0a, q0b, qpa, qpb;
    interp(K - 1, qma, qmb);
    interp(K, q0a, q0b);
    interp(K + 1, qpa, qpb);
    const float w = 1.0f / 64.0f;
    // the four fine rows of the next plane pair are loaded before the current
    // pair is corrected, so two pairs' loads are in flight
    float4 va = ld_f4(fine_u + idx), vb = ld_f4(fine_u + idx + nx);
    float4 vc = ld_f4(fine_u + idx + plane), vd = ld_f4(fine_u + idx + plane + nx);
    auto put = [&](float* p, float4 v, float4 a, float4 b) {      // p = v + (3 a + b) / 64
        v.x += (3.0f * a.x + b.x) * w;
        v.y += (3.0f * a.y + b.y) * w;
        v.z += (3.0f * a.z + b.z) * w;
        v.w += (3.0f * a.w + b.w) * w;
        *reinterpret_cast<float4*>(p) = v;
    };
    for (int k = k0; k < k1; k += 2, idx += 2 * plane) {
        float4 na = va, nb = vb, nc = vc, nd = vd;
        if (k + 2 < k1) {
            const int n = idx + 2 * plane;
            na = ld_f4(fine_u + n);
            nb = ld_f4(fine_u + n + nx);
            nc = ld_f4(fine_u + n + plane);
            nd = ld_f4(fine_u + n + plane + nx);
        }
        put(fine_u + idx, va, q0a, qma);
        put(fine_u + idx + nx, vb, q0b, qmb);
        put(fine_u + idx + plane, vc, q0a, qpa);
        put(fine_u + idx + plane + nx, vd, q0b, qpb);
        ++K;
        qma = q0a; qmb = q0b;
        q0a = qpa; q0b = qpb;
        if (k + 2 < k1) interp(K + 1, qpa, qpb);
        va = na; vb = nb; vc = nc; vd = nd;
    }
}

// ---------------------------------------------------------------------------
// Defect-correction update with the FP64 residual carried by recurrence.
// For phi <- phi + e (e: the FP32 correction of the inner V-cycle),
//   r = f - A phi   <-   r - A_0 e,
// where A_0 is the Laplacian with homogeneous ghosts (the Dirichlet data enter
// A affinely, so they cancel in A(phi + e) - A phi).  A_0 e is evaluated
// without rounding error that matters: the seven terms are summed in FP32
// with error-free transformations (TwoSum, and an FMA for the error of the
// product 6 e_c), giving hi + lo to about 2^-48 of the largest term; hi and lo
// then enter the FP64 residual with one FMA each.  Float <-> double
// conversions are done on the bit patterns (IEEE 754 fields, integer pipe):
// on GB300 every FP64-pipe instruction, conversions included, issues at 1/64
// of the FP32 rate, and this kernel keeps three of them per cell (phi + e and
// the two FMAs).
// ---------------------------------------------------------------------------
// r -= (A_0 e) for one cell, A_0 the homogeneous operator, formed without
// rounding: the FP32 neighbour sum is split by TwoSum into a value and its
// exact error (products by -6 and -2 are exact up to one FMA term), and both
// enter r through FP64 FMAs.
template <bool UNIFORM>
__device__ __forceinline__ double update_r(const LevelGeom& g, float c, float xm, float xp, float ym, float yp,
                                           float zm, float zp, double r) {
    if (UNIFORM) {
        // sum of the six neighbours minus 6 c, compensated
        const float p = -6.0f * c;
        const float perr = fmaf(-6.0f, c, -p);          // -6 c = p + perr exactly
        float s = xm, comp = perr, t;
        two_sum(s, xp, s, t); comp += t;
        two_sum(s, ym, s, t); comp += t;
        two_sum(s, yp, s, t); comp += t;
        two_sum(s, zm, s, t); comp += t;
        two_sum(s, zp, s, t); comp += t;
        two_sum(s, p, s, t); comp += t;
        const double nih2 = -g.ihx2;
        r = fma(nih2, f2d_bits(s), r);
        r = fma(nih2, f2d_bits(comp), r);
    } else {
        // per-axis second differences (-2 c is exact), compensated
        const float m2 = -2.0f * c;
        const float a[3][2] = {{xm, xp}, {ym, yp}, {zm, zp}};
        const double ih[3] = {g.ihx2, g.ihy2, g.ihz2};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float s, comp, t;
            two_sum(a[d][0], a[d][1], s, comp);
            two_sum(s, m2, s, t);
            comp += t;
            r = fma(-ih[d], f2d_bits(s), r);
            r = fma(-ih[d], f2d_bits(comp), r);
        }
    }
    return r;
}

template <bool UNIFORM>
__global__ void __launch_bounds__(BX * BY)
k_update_residual(const LevelGeom g, double* __restrict__ phi, const float* __restrict__ e,
                  double* __restrict__ r64, float* __restrict__ r32, Partial* partials, int kchunk) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    float sq = 0.0f, mx = 0.0f;
    if (i < g.nx && j < g.ny) {
        const int k0 = blockIdx.z * kchunk;
        const int k1 = min(k0 + kchunk, g.nz);
        const int plane = g.nx * g.ny;
        int idx = k0 * plane + j * g.nx + i;
        float c = e[idx];
        float zm = (k0 > 0) ? e[idx - plane] : z_low<false>(e, g, i, j, idx, plane, c);
        for (int k = k0; k < k1; ++k, idx += plane) {
            const float zp = (k < g.nz - 1) ? e[idx + plane] : z_high<false>(e, g, i, j, idx, plane, c);
            float xm, xp, ym, yp;
            xy_neighbours<false>(e, g, i, j, k, idx, c, xm, xp, ym, yp);
            const double r = update_r<UNIFORM>(g, c, xm, xp, ym, yp, zm, zp, r64[idx]);
            r64[idx] = r;
            phi[idx] = phi[idx] + f2d_bits(c);
            const float rf = d2f_bits(r);
            r32[idx] = rf;
            sq = fmaf(rf, rf, sq);
            mx = fmaxf(mx, fabsf(rf));
            zm = c;
            c = zp;
        }
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_reduce_write<float>(sq, mx, 0.0f, partials, bid);
}

// The same update on strips of four x cells (nx % 4 == 0, 16-byte aligned
// arrays): one 16-byte load of e per neighbour row and 16-byte loads and
// stores of phi and r, the z neighbours carried in registers, the z loop
// unrolled by two so the next plane's loads overlap the current arithmetic.

template <bool UNIFORM>
__global__ void __launch_bounds__(BX * BY, 4)
k_update_residual4(const LevelGeom g, double* __restrict__ phi, const float* __restrict__ e,
                   double* __restrict__ r64, float* __restrict__ r32, Partial* partials, int kchunk) {
    const int q = blockIdx.x * BX + threadIdx.x;        // strip: cells 4q .. 4q + 3
    const int j = blockIdx.y * BY + threadIdx.y;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    float sq = 0.0f, mx = 0.0f;
    if (4 * q < nx && j < ny) {
        const int i0 = 4 * q, plane = nx * ny;
        const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
        const int k0 = blockIdx.z * kchunk;
        const int k1 = min(k0 + kchunk, nz);
        int idx = k0 * plane + j * nx + i0;
        float4 c = ld_f4(e + idx);
        float4 zm = k0 > 0 ? ld_f4(e + idx - plane) : (pz ? ld_f4(e + idx + (nz - 1) * plane) : neg_f4(c));
#pragma unroll 1
        for (int k = k0; k < k1; ++k, idx += plane) {
            const float4 zp = k < nz - 1 ? ld_f4(e + idx + plane) : (pz ? ld_f4(e + idx - (nz - 1) * plane) : neg_f4(c));
            const float4 ym = j > 0 ? ld_f4(e + idx - nx) : (py ? ld_f4(e + idx + (ny - 1) * nx) : neg_f4(c));
            const float4 yp = j < ny - 1 ? ld_f4(e + idx + nx) : (py ? ld_f4(e + idx - (ny - 1) * nx) : neg_f4(c));
            const float xl = i0 > 0 ? e[idx - 1] : (px ? e[idx + nx - 1] : -c.x);
            const float xr = i0 + 4 < nx ? e[idx + 4] : (px ? e[idx + 4 - nx] : -c.w);
            double2 ra = ld_d2(r64 + idx), rb = ld_d2(r64 + idx + 2);
            double2 pa = ld_d2(phi + idx), pb = ld_d2(phi + idx + 2);
            ra.x = update_r<UNIFORM>(g, c.x, xl, c.y, ym.x, yp.x, zm.x, zp.x, ra.x);
            ra.y = update_r<UNIFORM>(g, c.y, c.x, c.z, ym.y, yp.y, zm.y, zp.y, ra.y);
            rb.x = update_r<UNIFORM>(g, c.z, c.y, c.w, ym.z, yp.z, zm.z, zp.z, rb.x);
            rb.y = update_r<UNIFORM>(g, c.w, c.z, xr, ym.w, yp.w, zm.w, zp.w, rb.y);
            *reinterpret_cast<double2*>(r64 + idx) = ra;
            *reinterpret_cast<double2*>(r64 + idx + 2) = rb;
            pa.x += f2d_bits(c.x);
            pa.y += f2d_bits(c.y);
            pb.x += f2d_bits(c.z);
            pb.y += f2d_bits(c.w);
            *reinterpret_cast<double2*>(phi + idx) = pa;
            *reinterpret_cast<double2*>(phi + idx + 2) = pb;
            const float4 rf = make_float4(d2f_bits(ra.x), d2f_bits(ra.y), d2f_bits(rb.x), d2f_bits(rb.y));
            *reinterpret_cast<float4*>(r32 + idx) = rf;
            sq = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, fmaf(rf.z, rf.z, fmaf(rf.w, rf.w, sq))));
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(rf.x), fabsf(rf.y)), fmaxf(fabsf(rf.z), fabsf(rf.w))));
            zm = c;
            c = zp;
        }
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_reduce_write<float>(sq, mx, 0.0f, partials, bid);
}

struct I4 {
    long long x, y, z, w;
};
__device__ __forceinline__ I4 fx_row(const double* p, unsigned M) {       // four cells, 16-byte aligned
    const double2 a = ld_d2(p), b = ld_d2(p + 2);
    return {fx_from(a.x, M), fx_from(a.y, M), fx_from(b.x, M), fx_from(b.y, M)};
}
__device__ __forceinline__ I4 fx_neg(const I4& c) { return {-c.x, -c.y, -c.z, -c.w}; }
// Dirichlet ghosts 2 phi_face - c of a strip whose four face values are
// consecutive (y and z walls); 2 phi_face on the scale of M is phi_face on
// the scale of M - 1.
__device__ __forceinline__ I4 fx_ghost_row(const double* face, const I4& c, unsigned M) {
    return {fx_from(face[0], M - 1u) - c.x, fx_from(face[1], M - 1u) - c.y, fx_from(face[2], M - 1u) - c.z,
            fx_from(face[3], M - 1u) - c.w};
}

// r = f - A phi of one cell from its integer neighbours.  Equal h: one exact
// integer sum S, rounded to FP64 by the hardware conversion, and
// r = f + coef S with coef = -ih2 2^(M - 1079) (a power-of-two scaling of
// ih2, so coef S is ih2 times the rounded sum exactly); otherwise the three
// axis sums, each rounded by fx_to_f64.
template <bool UNIFORM>
__device__ __forceinline__ double fx_cell(const LevelGeom& g, unsigned M, double coef, long long c, long long xm,
                                          long long xp, long long ym, long long yp, long long zm, long long zp,
                                          double f) {
    if (UNIFORM) return fma(coef, __ll2double_rn(((xm + xp) + (ym + yp)) + (zm + zp) - 6 * c), f);
    double r = fma(-g.ihx2, fx_to_f64((xm + xp) - 2 * c, M), f);
    r = fma(-g.ihy2, fx_to_f64((ym + yp) - 2 * c, M), r);
    return fma(-g.ihz2, fx_to_f64((zm + zp) - 2 * c, M), r);
}

// The largest biased exponent of the n FP64 values of u and, one above their
// own, of the Dirichlet face values of g, max-combined into *out.
__global__ void __launch_bounds__(256) k_max_exponent(const LevelGeom g, const double* __restrict__ u, long long n,
                                                      unsigned* out) {
    const long long tid = blockIdx.x * 256LL + threadIdx.x, stride = (long long)gridDim.x * 256LL;
    unsigned m = 0u;
    const uint4* v = reinterpret_cast<const uint4*>(u);   // two values per load (16-byte aligned)
    for (long long p = tid; p < n / 2; p += stride) {
        const uint4 w = v[p];
        m = max(m, max(w.y & 0x7ff00000u, w.w & 0x7ff00000u));
    }
    if (tid == 0 && (n & 1)) m = max(m, (unsigned)__double2hiint(u[n - 1]) & 0x7ff00000u);
    m >>= 20;
    for (int d = 0; d < 3; ++d) {
        if (g.per[d]) continue;
        const long long nf = d == 0 ? (long long)g.ny * g.nz : d == 1 ? (long long)g.nx * g.nz : (long long)g.nx * g.ny;
        for (int s = 0; s < 2; ++s) {
            const double* fc = g.face[2 * d + s];
            if (!fc) continue;
            for (long long p = tid; p < nf; p += stride)
                m = max(m, (((unsigned)__double2hiint(fc[p]) >> 20) & 0x7ffu) + 1u);
        }
    }
    __shared__ unsigned s_m[8];
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < 8 ? s_m[threadIdx.x] : 0u;
        m = __reduce_max_sync(0xffffffffu, m);
        if (threadIdx.x == 0) atomicMax(out, m);
    }
}

// Copies into shared memory that complete asynchronously (per thread, in
// commit groups).
__device__ __forceinline__ void cpa_copy16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cpa_copy8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_none() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Shared memory of k_residual_fx4: raw FP64 rows of a plane (the tile's BY
// rows and the rows j0 - 1, j0 + BY), its two x-halo cells per row and its f
// rows, in kFxSlots slots (plane p in slot p % kFxSlots, staged two planes
// ahead); the integer rows of two planes, with their x-halo cells.
constexpr int kFxTW = 4 * BX;                     // cells per tile row
constexpr int kFxSlots = 4;
struct FxSmem {
    double raw[kFxSlots][BY + 2][kFxTW];
    double rawx[kFxSlots][BY][2];
    double rawf[kFxSlots][BY][kFxTW];
    long long irow[2][BY + 2][kFxTW + 2];         // columns kFxTW, kFxTW + 1: the x-halo cells
};

__device__ __forceinline__ I4 fx_row_smem(const double* p, unsigned M) {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    return {fx_from(a.x, M), fx_from(a.y, M), fx_from(b.x, M), fx_from(b.y, M)};
}
__device__ __forceinline__ void fx_store_row(long long* d, const I4& v) {
    longlong2* q = reinterpret_cast<longlong2*>(d);
    q[0] = make_longlong2(v.x, v.y);
    q[1] = make_longlong2(v.z, v.w);
}
__device__ __forceinline__ I4 fx_load_row(const long long* s) {
    const longlong2 a = reinterpret_cast<const longlong2*>(s)[0], b = reinterpret_cast<const longlong2*>(s)[1];
    return {a.x, a.y, b.x, b.y};
}

// The residual on strips of four x cells (nx % 4 == 0, 16-byte aligned
// arrays): r into r64, its FP32 copy (truncated) into r32, the norms of the
// copy into partials; *mexp is the pre-pass's M.  A block owns a tile of
// 4 BX x BY cells and walks a z chunk.  The FP64 inputs of plane p (the
// tile's rows, the rows above and below it, the two x-halo cells of each row,
// the f rows) are copied into shared memory by cp.async two planes ahead; a
// thread converts its strip of plane p + 1 (its z neighbour above, kept in
// registers with the one below) and stores it as the integer row of that
// plane, the first and last warps convert the rows above and below the tile,
// and after one barrier per plane every thread reads its y neighbours from
// the integer rows, its x neighbours from the adjacent lanes (the halo cells
// at the tile's edges).  Cells at a wall or a periodic seam of the level take
// their neighbours directly (ghost rule or wrapped load).
template <bool UNIFORM, bool FACES>
__global__ void __launch_bounds__(BX * BY, 2)
k_residual_fx4(const LevelGeom g, const double* __restrict__ u, const double* __restrict__ rhs,
               float* __restrict__ r32, double* __restrict__ r64, Partial* partials, int kchunk,
               const unsigned* __restrict__ mexp) {
    extern __shared__ __align__(16) unsigned char fx_raw_smem[];
    FxSmem& S = *reinterpret_cast<FxSmem*>(fx_raw_smem);
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * BX + lane;
    const int it0 = blockIdx.x * kFxTW;                 // first cell of the tile row
    const int q = blockIdx.x * BX + lane;               // strip: cells 4q .. 4q + 3
    const int j0 = blockIdx.y * BY, j = j0 + w;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const unsigned M = *mexp;
    const bool act = 4 * q < nx && j < ny;
    const int i0 = 4 * q, plane = nx * ny;
    const int k0 = blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, nz);
    float sq = 0.0f, mx = 0.0f;
    auto out = [&](int at, double ra, double rb, double rc, double rd) {
        *reinterpret_cast<double2*>(r64 + at) = make_double2(ra, rb);
        *reinterpret_cast<double2*>(r64 + at + 2) = make_double2(rc, rd);
        const float4 rf = make_float4(d2f_bits(ra), d2f_bits(rb), d2f_bits(rc), d2f_bits(rd));
        *reinterpret_cast<float4*>(r32 + at) = rf;
        sq = fmaf(rf.x, rf.x, fmaf(rf.y, rf.y, fmaf(rf.z, rf.z, fmaf(rf.w, rf.w, sq))));
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(rf.x), fabsf(rf.y)), fmaxf(fabsf(rf.z), fabsf(rf.w))));
    };
    if (M < kFxMinExp || M > kFxMaxExp) {
        // beyond the fixed-point scale's range, or not finite: the FP64 stencil
        if (act) {
            int idx = k0 * plane + j * nx + i0;
#pragma unroll 1
            for (int k = k0; k < k1; ++k, idx += plane) {
                double r[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) r[t] = rhs[idx + t] - lap_at<FACES, double>(u, g, i0 + t, j, k);
                out(idx, r[0], r[1], r[2], r[3]);
            }
        }
    } else {
        const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
        const double* fxm = FACES && !px ? g.face[0] : nullptr;
        const double* fxp = FACES && !px ? g.face[1] : nullptr;
        const double* fym = FACES && !py ? g.face[2] : nullptr;
        const double* fyp = FACES && !py ? g.face[3] : nullptr;
        const double* fzm = FACES && !pz ? g.face[4] : nullptr;
        const double* fzp = FACES && !pz ? g.face[5] : nullptr;
        // equal h: S 2^(M - 1079) ih2 = S coef, the scale folded into one FP64 coefficient
        const double coef = -g.ihx2 * __longlong_as_double((long long)(M - 56u) << 52);
        // This thread's copies of a plane: two FP64 cells (16 bytes) of column
        // cx of the rows cr, cr + 4, cr + 8 of the raw rows (row r is level
        // row j0 - 1 + r) and of the rows cr, cr + 4 of the f rows, each only
        // inside the level; threads of warp kFxHaloWarp copy the x-halo cells.
        constexpr int kRowChunks = kFxTW / 2, kThreads = BX * BY;
        static_assert(kThreads == 4 * kRowChunks && BY == 8, "the copy pattern assumes 256 threads and 8 rows");
        constexpr int kFxHaloWarp = BY / 2;
        const int cx = 2 * (tid % kRowChunks), cr = tid / kRowChunks;
        const bool col_in = it0 + cx < nx;
        const int hx_t = tid - kFxHaloWarp * BX;                                // x-halo duty: 0 .. 2 BY - 1
        const int hx_r = hx_t >> 1, hx_side = hx_t & 1;
        const int hx_i = hx_side ? it0 + kFxTW : it0 - 1;
        const bool hx_in = hx_t >= 0 && hx_t < 2 * BY && j0 + hx_r < ny && hx_i >= 0 && hx_i < nx;
        const int hx_off = (j0 + hx_r) * nx + hx_i;
        auto stage = [&](int p) {
            // plane 0 for p = nz on a periodic z axis; nothing beyond a z wall
            const int ps = p < nz ? p : (pz ? 0 : -1);
            if (ps < 0) return;
            const int sl = p % kFxSlots;
            const double* ub = u + (long long)ps * plane + it0 + cx;
            const double* fb = rhs + (long long)ps * plane + it0 + cx;
            if (col_in) {
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const int r = cr + 4 * t, jj = j0 - 1 + r;
                    if (r < BY + 2 && jj >= 0 && jj < ny) cpa_copy16(&S.raw[sl][r][cx], ub + jj * nx);
                }
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int r = cr + 4 * t;
                    if (j0 + r < ny) cpa_copy16(&S.rawf[sl][r][cx], fb + (j0 + r) * nx);
                }
            }
            if (hx_in) cpa_copy8(&S.rawx[sl][hx_r][hx_side], u + (long long)ps * plane + hx_off);
        };
        // the integer row of plane p: own strip (the caller's value), the rows
        // above and below the tile and the x-halo cells from the staged copies
        auto put_rows = [&](int p, const I4& own) {
            long long(*ir)[kFxTW + 2] = S.irow[p & 1];
            const int sl = p % kFxSlots;
            if (act) fx_store_row(&ir[w + 1][4 * lane], own);
            if (w == 0 && act && j0 > 0) fx_store_row(&ir[0][4 * lane], fx_row_smem(&S.raw[sl][0][4 * lane], M));
            if (w == BY - 1 && act && j0 + BY < ny)
                fx_store_row(&ir[BY + 1][4 * lane], fx_row_smem(&S.raw[sl][BY + 1][4 * lane], M));
            if (hx_in) ir[hx_r + 1][kFxTW + hx_side] = fx_from(S.rawx[sl][hx_r][hx_side], M);
        };
        const int idx0 = act ? j * nx + i0 : 0;
        I4 c = {0, 0, 0, 0}, zm = {0, 0, 0, 0};
        stage(k0);
        cpa_commit_group();
        if (k0 + 1 <= k1) stage(k0 + 1);
        cpa_commit_group();
        cpa_wait_but_one();
        __syncthreads();
        if (act) {
            c = fx_row_smem(&S.raw[k0 % kFxSlots][w + 1][4 * lane], M);
            const int at = k0 * plane + idx0;
            zm = k0 > 0 ? fx_row(u + at - plane, M)
                        : (pz ? fx_row(u + at + (nz - 1) * plane, M)
                              : (fzm ? fx_ghost_row(fzm + j * nx + i0, c, M) : fx_neg(c)));
        }
        put_rows(k0, c);
#pragma unroll 1
        for (int k = k0; k < k1; ++k) {
            if (k + 2 <= k1) stage(k + 2);
            cpa_commit_group();
            cpa_wait_but_one();                        // this thread's copies of plane k + 1 have landed
            __syncthreads();                           // everyone's; the integer rows of plane k are complete
            const int at = k * plane + idx0;
            I4 zp = {0, 0, 0, 0};
            if (act) {
                zp = (k + 1 < nz || pz) ? fx_row_smem(&S.raw[(k + 1) % kFxSlots][w + 1][4 * lane], M)
                                        : (fzp ? fx_ghost_row(fzp + j * nx + i0, c, M) : fx_neg(c));
            }
            long long xl = __shfl_up_sync(0xffffffffu, c.w, 1);
            long long xr = __shfl_down_sync(0xffffffffu, c.x, 1);
            if (act) {
                const int sl = k % kFxSlots;
                const long long(*ir)[kFxTW + 2] = S.irow[k & 1];
                if (lane == 0)
                    xl = i0 > 0 ? ir[w + 1][kFxTW]
                                : (px ? fx_from(u[at + nx - 1], M)
                                      : (fxm ? fx_from(fxm[k * ny + j], M - 1u) - c.x : -c.x));
                if (i0 + 4 >= nx)
                    xr = px ? fx_from(u[at + 4 - nx], M) : (fxp ? fx_from(fxp[k * ny + j], M - 1u) - c.w : -c.w);
                else if (lane == BX - 1)
                    xr = ir[w + 1][kFxTW + 1];
                const I4 ym = j > 0 ? fx_load_row(&ir[w][4 * lane])
                                    : (py ? fx_row(u + at + (ny - 1) * nx, M)
                                          : (fym ? fx_ghost_row(fym + k * nx + i0, c, M) : fx_neg(c)));
                const I4 yp = j < ny - 1 ? fx_load_row(&ir[w + 2][4 * lane])
                                         : (py ? fx_row(u + at - (ny - 1) * nx, M)
                                               : (fyp ? fx_ghost_row(fyp + k * nx + i0, c, M) : fx_neg(c)));
                const double2 fa = *reinterpret_cast<const double2*>(&S.rawf[sl][w][4 * lane]);
                const double2 fb = *reinterpret_cast<const double2*>(&S.rawf[sl][w][4 * lane + 2]);
                out(at, fx_cell<UNIFORM>(g, M, coef, c.x, xl, c.y, ym.x, yp.x, zm.x, zp.x, fa.x),
                    fx_cell<UNIFORM>(g, M, coef, c.y, c.x, c.z, ym.y, yp.y, zm.y, zp.y, fa.y),
                    fx_cell<UNIFORM>(g, M, coef, c.z, c.y, c.w, ym.z, yp.z, zm.z, zp.z, fb.x),
                    fx_cell<UNIFORM>(g, M, coef, c.w, c.z, xr, ym.w, yp.w, zm.w, zp.w, fb.y));
            }
            if (k + 1 < k1) put_rows(k + 1, zp);
            zm = c;
            c = zp;
        }
        cpa_wait_none();
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_reduce_write<float>(sq, mx, 0.0f, partials, bid);
}

// Shared memory of k_gravity_fx4: the FP64 rows j0 - 2 .. j0 + BY + 1 of a
// staged plane and its x-halo cells (it0 - 2, it0 - 1, it0 + TW, it0 + TW + 1)
// in kGvSlots slots (plane p in slot p % kGvSlots, staged three planes
// ahead), and the integer rows of two planes with their x-halo cells.
constexpr int kGvSlots = 4;
struct GvSmem {
    double raw[kGvSlots][BY + 4][kFxTW];
    double rawx[kGvSlots][BY][4];
    long long irow[2][BY + 4][kFxTW + 4];
};

// The acceleration on strips of four x cells (nx % 4 == 0, 16-byte aligned phi
// and out), every component's combination exact in fixed point on the scale of
// *mexp (GravFx); a scale out of range falls back to FP64 per cell.  A block
// owns a 4 BX x BY tile and walks its z chunk; the plane's rows (with two halo
// rows on each side) and x-halo cells are copied into shared memory by
// cp.async three planes ahead.  A thread converts its strip of plane k + 2
// once and keeps planes k - 2 .. k + 2 of it in registers; it stores plane
// k + 1's strip as that plane's integer row, the first two and last two warps
// convert the halo rows, one warp the x-halo cells; after one barrier per
// plane the y neighbours come from the integer rows, the x neighbours from
// the adjacent lanes.  Neighbours past a Dirichlet wall are 2 phi_face - the
// mirror cell (two ghost layers; at least two cells on such an axis), past a
// periodic seam the wrapped cells (loaded directly).
__global__ void __launch_bounds__(BX * BY, 2)
k_gravity_fx4(const LevelGeom g, const double* __restrict__ u, double* __restrict__ out, double cx, double cy,
              double cz, int kchunk, const unsigned* __restrict__ mexp) {
    extern __shared__ __align__(16) unsigned char gv_raw_smem[];
    GvSmem& S = *reinterpret_cast<GvSmem*>(gv_raw_smem);
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * BX + lane;
    const int it0 = blockIdx.x * kFxTW;                 // first cell of the tile row
    const int q = blockIdx.x * BX + lane;               // strip: cells 4q .. 4q + 3
    const int j0 = blockIdx.y * BY, j = j0 + w;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const unsigned M = *mexp;
    const bool xin = 4 * q < nx;
    const bool act = xin && j < ny;
    const int i0 = 4 * q, plane = nx * ny;
    const long long n = (long long)plane * nz;
    const int k0 = blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, nz);
    auto store = [&](long long at, const double (&r)[3][4]) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            *reinterpret_cast<double2*>(out + d * n + at) = make_double2(r[d][0], r[d][1]);
            *reinterpret_cast<double2*>(out + d * n + at + 2) = make_double2(r[d][2], r[d][3]);
        }
    };
    if (M < kFxMinExp || M > kFxMaxExp) {
        // beyond the fixed-point scale's range, or not finite: FP64 per cell
        if (act) {
            const GravF64 pv{};
#pragma unroll 1
            for (int k = k0; k < k1; ++k) {
                double r[3][4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int i = i0 + t, col = j * nx + i;
                    r[0][t] = pv.comp(cx, halo_phi(u, g, i + 1, j, k, pv), halo_phi(u, g, i - 1, j, k, pv),
                                      halo_phi(u, g, i + 2, j, k, pv), halo_phi(u, g, i - 2, j, k, pv));
                    r[1][t] = pv.comp(cy, halo_phi(u, g, i, j + 1, k, pv), halo_phi(u, g, i, j - 1, k, pv),
                                      halo_phi(u, g, i, j + 2, k, pv), halo_phi(u, g, i, j - 2, k, pv));
                    r[2][t] = pv.comp(cz, zcol_phi(u, g, col, col, k + 1, pv), zcol_phi(u, g, col, col, k - 1, pv),
                                      zcol_phi(u, g, col, col, k + 2, pv), zcol_phi(u, g, col, col, k - 2, pv));
                }
                store((long long)k * plane + j * nx + i0, r);
            }
        }
        return;
    }
    const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
    const double* fxm = !px ? g.face[0] : nullptr;
    const double* fxp = !px ? g.face[1] : nullptr;
    const double* fym = !py ? g.face[2] : nullptr;
    const double* fyp = !py ? g.face[3] : nullptr;
    const double* fzm = !pz ? g.face[4] : nullptr;
    const double* fzp = !pz ? g.face[5] : nullptr;
    // 2 phi_face - mirror (zero face values without data)
    auto ghost1 = [&](const double* f, int at, long long mirror) {
        return (f ? fx_from(f[at], M - 1u) : 0LL) - mirror;
    };
    auto ghost4 = [&](const double* f, int at, const I4& m) -> I4 {
        return {ghost1(f, at, m.x), ghost1(f, at + 1, m.y), ghost1(f, at + 2, m.z), ghost1(f, at + 3, m.w)};
    };
    // this thread's copies of a plane: 16 bytes of column cx of the raw rows
    // cr, cr + 4, cr + 8 (row r is level row j0 - 2 + r), inside the level;
    // warp kGvHaloWarp copies the x-halo cells
    constexpr int kRowChunks = kFxTW / 2;
    static_assert(BX * BY == 4 * kRowChunks && BY == 8, "the copy pattern assumes 256 threads and 8 rows");
    constexpr int kGvHaloWarp = BY / 2;
    const int cx2 = 2 * (tid % kRowChunks), cr = tid / kRowChunks;
    const bool col_in = it0 + cx2 < nx;
    const int hx_r = lane >> 2, hx_side = lane & 3;                        // warp kGvHaloWarp: 8 rows x 4 cells
    const int hx_i = hx_side < 2 ? it0 - 2 + hx_side : it0 + kFxTW + (hx_side - 2);
    const bool hx_in = w == kGvHaloWarp && j0 + hx_r < ny && hx_i >= 0 && hx_i < nx;
    const int hx_off = (j0 + hx_r) * nx + hx_i;
    auto stage = [&](int p) {
        const int ps = p < nz ? p : (pz ? p % nz : -1);                     // past the top: wrapped (nz may be 1), or nothing
        if (ps < 0) return;
        const int sl = p % kGvSlots;
        const double* ub = u + (long long)ps * plane + it0 + cx2;
        if (col_in) {
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int r = cr + 4 * t, jj = j0 - 2 + r;
                if (jj >= 0 && jj < ny) cpa_copy16(&S.raw[sl][r][cx2], ub + jj * nx);
            }
        }
        if (hx_in) cpa_copy8(&S.rawx[sl][hx_r][hx_side], u + (long long)ps * plane + hx_off);
    };
    // the integer row of plane p: own strip (the caller's value), the two halo
    // rows on each side of the tile and the x-halo cells from the staged copies
    auto put_rows = [&](int p, const I4& own) {
        long long(*ir)[kFxTW + 4] = S.irow[p & 1];
        const int sl = p % kGvSlots;
        if (act) fx_store_row(&ir[w + 2][4 * lane], own);
        if (xin) {
            if (w < 2 && j0 - 2 + w >= 0)
                fx_store_row(&ir[w][4 * lane], fx_row_smem(&S.raw[sl][w][4 * lane], M));
            if (w >= BY - 2 && j0 + w + 2 < ny)
                fx_store_row(&ir[w + 4][4 * lane], fx_row_smem(&S.raw[sl][w + 4][4 * lane], M));
        }
        if (hx_in) ir[hx_r + 2][kFxTW + hx_side] = fx_from(S.rawx[sl][hx_r][hx_side], M);
    };
    const int idx0 = act ? j * nx + i0 : 0;
    // own strip at plane p straight from memory (the chunk's first planes)
    auto own_direct = [&](int p) -> I4 {
        if (p >= 0 && p < nz) return fx_row(u + (long long)p * plane + idx0, M);
        if (pz) return fx_row(u + (long long)((p % nz + nz) % nz) * plane + idx0, M);
        const int m = p < 0 ? -1 - p : 2 * nz - 1 - p;
        return ghost4(p < 0 ? fzm : fzp, j * nx + i0, fx_row(u + (long long)m * plane + idx0, M));
    };
    stage(k0);
    cpa_commit_group();
    stage(k0 + 1);
    cpa_commit_group();
    if (k0 + 2 <= k1 + 1) stage(k0 + 2);
    cpa_commit_group();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");     // planes k0 and k0 + 1 have landed
    __syncthreads();
    I4 zm2 = {0, 0, 0, 0}, zm1 = zm2, c = zm2, zp1 = zm2;
    if (act) {
        c = fx_row_smem(&S.raw[k0 % kGvSlots][2 + w][4 * lane], M);
        zp1 = (k0 + 1 < nz || pz) ? fx_row_smem(&S.raw[(k0 + 1) % kGvSlots][2 + w][4 * lane], M)
                                  : ghost4(fzp, j * nx + i0, c);
        zm1 = own_direct(k0 - 1);
        zm2 = own_direct(k0 - 2);
    }
    put_rows(k0, c);
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
        if (k + 3 <= k1 + 1) stage(k + 3);
        cpa_commit_group();
        cpa_wait_but_one();                           // this thread's copies of plane k + 2 have landed
        __syncthreads();                              // everyone's; the integer rows of plane k are complete
        const long long at = (long long)k * plane + idx0;
        I4 zp2 = {0, 0, 0, 0};
        if (act) {
            if (k + 2 < nz || pz) zp2 = fx_row_smem(&S.raw[(k + 2) % kGvSlots][2 + w][4 * lane], M);
            else zp2 = ghost4(fzp, j * nx + i0, k + 2 == nz ? zp1 : zm1);   // mirrors of planes nz, nz + 1
        }
        const long long l1 = __shfl_up_sync(0xffffffffu, c.w, 1), l2 = __shfl_up_sync(0xffffffffu, c.z, 1);
        const long long r1 = __shfl_down_sync(0xffffffffu, c.x, 1), r2 = __shfl_down_sync(0xffffffffu, c.y, 1);
        if (act) {
            const long long(*ir)[kFxTW + 4] = S.irow[k & 1];
            long long X[8] = {l2, l1, c.x, c.y, c.z, c.w, r1, r2};        // cells i0 - 2 .. i0 + 5
            if (lane == 0) {
                if (i0 > 0) {
                    X[0] = ir[w + 2][kFxTW];
                    X[1] = ir[w + 2][kFxTW + 1];
                } else if (px) {
                    X[0] = fx_from(u[at + nx - 2], M);
                    X[1] = fx_from(u[at + nx - 1], M);
                } else {
                    X[0] = ghost1(fxm, k * ny + j, c.y);
                    X[1] = ghost1(fxm, k * ny + j, c.x);
                }
            }
            if (i0 + 4 >= nx) {
                if (px) {
                    X[6] = fx_from(u[at + 4 - nx], M);
                    X[7] = fx_from(u[at + 5 - nx], M);
                } else {
                    X[6] = ghost1(fxp, k * ny + j, c.w);
                    X[7] = ghost1(fxp, k * ny + j, c.z);
                }
            } else if (lane == BX - 1) {
                X[6] = ir[w + 2][kFxTW + 2];
                X[7] = ir[w + 2][kFxTW + 3];
            }
            // rows j - 2, j - 1, j + 1, j + 2
            I4 Y[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int d = e < 2 ? e - 2 : e - 1, r = j + d;
                if (r >= 0 && r < ny) {
                    Y[e] = fx_load_row(&ir[w + 2 + d][4 * lane]);
                } else if (py) {
                    Y[e] = fx_row(u + (long long)k * plane + (long long)(r < 0 ? r + ny : r - ny) * nx + i0, M);
                } else {
                    const int m = r < 0 ? -1 - r : 2 * ny - 1 - r;             // the mirror row, staged
                    Y[e] = ghost4(r < 0 ? fym : fyp, k * nx + i0, fx_load_row(&ir[m - j0 + 2][4 * lane]));
                }
            }
            // one component at a time, stored as it is formed
            const GravFx pv{M};
            double* o = out + at;
            *reinterpret_cast<double2*>(o) = make_double2(pv.comp(cx, X[3], X[1], X[4], X[0]),
                                                          pv.comp(cx, X[4], X[2], X[5], X[1]));
            *reinterpret_cast<double2*>(o + 2) = make_double2(pv.comp(cx, X[5], X[3], X[6], X[2]),
                                                              pv.comp(cx, X[6], X[4], X[7], X[3]));
            o += n;
            *reinterpret_cast<double2*>(o) = make_double2(pv.comp(cy, Y[2].x, Y[1].x, Y[3].x, Y[0].x),
                                                          pv.comp(cy, Y[2].y, Y[1].y, Y[3].y, Y[0].y));
            *reinterpret_cast<double2*>(o + 2) = make_double2(pv.comp(cy, Y[2].z, Y[1].z, Y[3].z, Y[0].z),
                                                              pv.comp(cy, Y[2].w, Y[1].w, Y[3].w, Y[0].w));
            o += n;
            *reinterpret_cast<double2*>(o) = make_double2(pv.comp(cz, zp1.x, zm1.x, zp2.x, zm2.x),
                                                          pv.comp(cz, zp1.y, zm1.y, zp2.y, zm2.y));
            *reinterpret_cast<double2*>(o + 2) = make_double2(pv.comp(cz, zp1.z, zm1.z, zp2.z, zm2.z),
                                                              pv.comp(cz, zp1.w, zm1.w, zp2.w, zm2.w));
        }
        if (k + 1 < k1) put_rows(k + 1, zp1);
        zm2 = zm1;
        zm1 = c;
        c = zp1;
        zp1 = zp2;
    }
    cpa_wait_none();
}

// ---------------------------------------------------------------------------
// Small helpers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRedThreads) k_finalize(const Partial* __restrict__ p, int n,
                                                          Reduced* out) {
    // Fixed order (deterministic): thread t folds partials t, t + 256, ...
    // four at a time so that their loads are in flight together, then the
    // warps fold by shuffles and warp 0 folds the eight warp results.
    __shared__ double s_sq[kRedThreads / 32], s_mx[kRedThreads / 32], s_sum[kRedThreads / 32];
    double sq = 0.0, mx = 0.0, sm = 0.0;
    int t = threadIdx.x;
    for (; t + 3 * kRedThreads < n; t += 4 * kRedThreads) {
        Partial a[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) a[e] = p[t + e * kRedThreads];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            sq += a[e].sumsq;
            mx = fmax(mx, a[e].maxabs);
            sm += a[e].sum;
        }
    }
    for (; t < n; t += kRedThreads) {
        sq += p[t].sumsq;
        mx = fmax(mx, p[t].maxabs);
        sm += p[t].sum;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sq += __shfl_down_sync(0xffffffffu, sq, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        sm += __shfl_down_sync(0xffffffffu, sm, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_sq[w] = sq;
        s_mx[w] = mx;
        s_sum[w] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = s_sq[0], b = s_mx[0], c = s_sum[0];
        for (int k = 1; k < kRedThreads / 32; ++k) {
            a += s_sq[k];
            b = fmax(b, s_mx[k]);
            c += s_sum[k];
        }
        out->sumsq = a;
        out->maxabs = b;
        out->sum = c;
        out->count = double(n);
    }
}

template <typename T>
__global__ void k_subtract_mean(T* x, long long n, const Reduced* red) {
    const T mean = T(red->sum) / T(n);            // in T: no FP64 division in FP32 kernels
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        x[t] = x[t] - mean;
}

__global__ void k_scale_copy(const double* src, double* dst, double scale, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        dst[t] = scale * src[t];
}

// Copies over the CPU-GPU link: one side is pinned host memory mapped into
// the device address space.  16-byte accesses with four in flight per thread
// keep enough bytes outstanding to cover the link's latency.
template <bool SCALE>
__global__ void __launch_bounds__(256) k_link_copy(const double2* __restrict__ src, double2* __restrict__ dst,
                                                   double scale, long long n2) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; t + 3 * stride < n2; t += 4 * stride) {
        double2 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = src[t + i * stride];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (SCALE) {
                v[i].x = scale * v[i].x;
                v[i].y = scale * v[i].y;
            }
            dst[t + i * stride] = v[i];
        }
    }
    for (; t < n2; t += stride) {
        double2 v = src[t];
        if (SCALE) {
            v.x = scale * v.x;
            v.y = scale * v.y;
        }
        dst[t] = v;
    }
}

__global__ void k_add_f32_to_f64(double* phi, const float* __restrict__ e, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        phi[t] = phi[t] + double(e[t]);
}

__global__ void __launch_bounds__(256) k_sum_f64(const double* __restrict__ x, long long n,
                                                 Partial* partials) {
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        s += x[t];
    block_reduce_write<double>(0.0, 0.0, s, partials, blockIdx.x);
}

int grid1d(long long n) {
    long long b = (n + 255) / 256;
    if (b > kSumBlocks) b = kSumBlocks;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
long long residual_blocks(const LevelGeom& g) {
    const int kc = kchunk_for(g, BX, BY);
    return (long long)((g.nx + BX - 1) / BX) * ((g.ny + BY - 1) / BY) * ((g.nz + kc - 1) / kc);
}

long long residual_zero_blocks(const LevelGeom& g) {
    const int kc = kchunk_for(g, 4 * BX, BY);
    const long long strips = (long long)((g.nx / 4 + BX - 1) / BX) * ((g.ny + BY - 1) / BY) * ((g.nz + kc - 1) / kc);
    return std::max(residual_blocks(g), strips + kWallBlocks);
}

// SMs of the current device (queried once).
long long sm_count() {
    static const long long n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || v <= 0) {
            cudaGetLastError();
            return 152LL;
        }
        return (long long)v;
    }();
    return n;
}

long long restrict_blocks(const LevelGeom& g) {
    if (g.twod) return (long long)((g.nx + BX - 1) / BX) * ((g.ny + BY - 1) / BY);
    const int kc = even_kchunk(g);
    return (long long)((g.nx + BX - 1) / BX) * ((g.ny + BY - 1) / BY) * ((g.nz + kc - 1) / kc);
}

bool has_faces(const LevelGeom& g) {
    for (int f = 0; f < 6; ++f)
        if (g.face[f]) return true;
    return false;
}

template <typename T, int ORDER, bool FIRST>
void launch_stage_f(bool faces, dim3 grid, dim3 block, cudaStream_t st, const LevelGeom& g, const CoefT<T>& cf,
                    const T* ym1, const T* ym2, const T* y0, const T* z0, const T* rhs, T* out, T* z0_out, int kc) {
    if (faces) k_stage<T, ORDER, FIRST, true><<<grid, block, 0, st>>>(g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
    else k_stage<T, ORDER, FIRST, false><<<grid, block, 0, st>>>(g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
}

template <typename T>
cudaError_t launch_stage(const LevelGeom& g, int order, bool first, const StageCoef& c,
                         const T* ym1, const T* ym2, const T* y0, const T* z0, const T* rhs,
                         T* out, T* z0_out, cudaStream_t st) {
    CoefT<T> cf;
    cf.tau = T(c.tau); cf.mut1 = T(c.mut1); cf.mu = T(c.mu); cf.nu = T(c.nu);
    cf.mut_tau = T(c.mut_tau); cf.c0 = T(c.c0); cf.gt = T(c.gt);
    const bool faces = has_faces(g);
    if constexpr (std::is_same<T, float>::value) {
        const uintptr_t al = reinterpret_cast<uintptr_t>(ym1) | reinterpret_cast<uintptr_t>(ym2) |
                             reinterpret_cast<uintptr_t>(y0) | reinterpret_cast<uintptr_t>(z0) |
                             reinterpret_cast<uintptr_t>(rhs) | reinterpret_cast<uintptr_t>(out) |
                             reinterpret_cast<uintptr_t>(z0_out);
        if (!faces && (g.nx & 3) == 0 && (al & 15) == 0) {
            // strips: a block of 32 x 8 strips, or 16 x 16 where a row holds 16 strips or fewer
            const int bx = g.nx / 4 <= 16 ? 16 : BX, by = BX * BY / bx;
            const int kc = kchunk_for(g, 4 * bx, by);
            dim3 block(bx, by, 1);
            dim3 grid((g.nx / 4 + bx - 1) / bx, (g.ny + by - 1) / by, (g.nz + kc - 1) / kc);
            if (order == 1) {
                if (first) k_stage4<1, true><<<grid, block, 0, st>>>(g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
                else k_stage4<1, false><<<grid, block, 0, st>>>(g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
            } else {
                if (first) k_stage4<2, true><<<grid, block, 0, st>>>(g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
                else k_stage4<2, false><<<grid, block, 0, st>>>(g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
            }
            return cudaGetLastError();
        }
    }
    const int kc = kchunk_for(g, BX, BY);
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kc - 1) / kc);
    if (order == 1) {
        if (first) launch_stage_f<T, 1, true>(faces, grid, block, st, g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
        else launch_stage_f<T, 1, false>(faces, grid, block, st, g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
    } else {
        if (first) launch_stage_f<T, 2, true>(faces, grid, block, st, g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
        else launch_stage_f<T, 2, false>(faces, grid, block, st, g, cf, ym1, ym2, y0, z0, rhs, out, z0_out, kc);
    }
    return cudaGetLastError();
}

template <typename TO>
cudaError_t launch_residual_zero(const LevelGeom& g, const double* rhs, TO* r_out, Partial* partials,
                                 int* nblocks_out, cudaStream_t st, double* r_full, int* nkernels) {
    if (nkernels) *nkernels = 1;
    if constexpr (std::is_same<TO, float>::value) {
        const bool aligned = ((reinterpret_cast<uintptr_t>(rhs) | reinterpret_cast<uintptr_t>(r_out) |
                               reinterpret_cast<uintptr_t>(r_full)) & 15) == 0;
        if ((g.nx & 3) == 0 && aligned) {
            const int kc = kchunk_for(g, 4 * BX, BY);
            dim3 block(BX, BY, 1);
            dim3 grid((unsigned)((g.nx / 4 + BX - 1) / BX), (unsigned)((g.ny + BY - 1) / BY),
                      (unsigned)((g.nz + kc - 1) / kc));
            const int nb = (int)(grid.x * grid.y * grid.z);
            k_residual_zero4<<<grid, block, 0, st>>>(g, rhs, r_out, r_full, partials, kc);
            int nw = 0;
            if (has_faces(g)) {
                nw = kWallBlocks;
                const bool uniform = g.ihx2 == g.ihy2 && g.ihy2 == g.ihz2;
                if (uniform) k_residual_zero_walls<true><<<nw, block, 0, st>>>(g, rhs, r_out, r_full, partials + nb);
                else k_residual_zero_walls<false><<<nw, block, 0, st>>>(g, rhs, r_out, r_full, partials + nb);
            }
            if (nblocks_out) *nblocks_out = nb + nw;
            if (nkernels) *nkernels = nw > 0 ? 2 : 1;
            return cudaGetLastError();
        }
    }
    const int kc = kchunk_for(g, BX, BY);                        // the blocks of launch_residual
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kc - 1) / kc);
    const bool uniform = g.ihx2 == g.ihy2 && g.ihy2 == g.ihz2;
    const bool faces = has_faces(g);
    if (uniform && faces) k_residual_zero<TO, true, true><<<grid, block, 0, st>>>(g, rhs, r_out, r_full, partials, kc);
    else if (uniform) k_residual_zero<TO, true, false><<<grid, block, 0, st>>>(g, rhs, r_out, r_full, partials, kc);
    else if (faces) k_residual_zero<TO, false, true><<<grid, block, 0, st>>>(g, rhs, r_out, r_full, partials, kc);
    else k_residual_zero<TO, false, false><<<grid, block, 0, st>>>(g, rhs, r_out, r_full, partials, kc);
    if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
    return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_residual(const LevelGeom& g, const TI* u, const TI* rhs, TO* r_out,
                            Partial* partials, int* nblocks_out, cudaStream_t st, TI* r_full) {
    const int kc = kchunk_for(g, BX, BY);
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kc - 1) / kc);
    const bool uniform = g.ihx2 == g.ihy2 && g.ihy2 == g.ihz2;   // (also true for the FP32 copies)
    const bool faces = has_faces(g);
    if (uniform && faces) k_residual<TI, TO, true, true><<<grid, block, 0, st>>>(g, u, rhs, r_out, r_full, partials, kc);
    else if (uniform) k_residual<TI, TO, true, false><<<grid, block, 0, st>>>(g, u, rhs, r_out, r_full, partials, kc);
    else if (faces) k_residual<TI, TO, false, true><<<grid, block, 0, st>>>(g, u, rhs, r_out, r_full, partials, kc);
    else k_residual<TI, TO, false, false><<<grid, block, 0, st>>>(g, u, rhs, r_out, r_full, partials, kc);
    if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_restrict(const LevelGeom& g, const T* u, const T* rhs, T* coarse_out,
                                     Partial* partials, int* nblocks_out, cudaStream_t st) {
    if (g.twod) {
        dim3 block(BX, BY, 1);
        dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, 1);
        if (has_faces(g)) k_residual_restrict2d<T, true><<<grid, block, 0, st>>>(g, u, rhs, coarse_out, partials);
        else k_residual_restrict2d<T, false><<<grid, block, 0, st>>>(g, u, rhs, coarse_out, partials);
        if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y);
        return cudaGetLastError();
    }
    if constexpr (std::is_same<T, float>::value) {
        const bool aligned = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(rhs) |
                               reinterpret_cast<uintptr_t>(coarse_out)) & 15) == 0;
        if (!has_faces(g) && (g.nx & 3) == 0 && (g.ny & 1) == 0 && (g.nz & 1) == 0 && aligned) {
            // as many blocks as the scalar launch at most (the partials buffer)
            const long long gx = (g.nx / 4 + BX - 1) / BX, gy = (g.ny / 2 + BY - 1) / BY;
            const long long chunks = std::min<long long>(g.nz / 2, std::max(1LL, restrict_blocks(g) / (gx * gy)));
            int kc = (int)((g.nz + chunks - 1) / chunks);
            kc += kc & 1;
            // longer z chunks re-read fewer halo planes: up to 16 planes while
            // the launch keeps three blocks per SM (256^3: 25 against 32 us)
            while (kc < 16 && gx * gy * ((g.nz + 2 * kc - 1) / (2 * kc)) >= 3LL * sm_count()) kc *= 2;
            dim3 block(BX, BY, 1);
            dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)((g.nz + kc - 1) / kc));
            k_residual_restrict4<<<grid, block, 0, st>>>(g, u, rhs, coarse_out, partials, kc);
            if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
            return cudaGetLastError();
        }
    }
    const int kc = even_kchunk(g);
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kc - 1) / kc);
    if (has_faces(g)) k_residual_restrict<T, true><<<grid, block, 0, st>>>(g, u, rhs, coarse_out, partials, kc);
    else k_residual_restrict<T, false><<<grid, block, 0, st>>>(g, u, rhs, coarse_out, partials, kc);
    if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_correct(const LevelGeom& g, const T* coarse, T* fine_u, cudaStream_t st) {
    if (g.twod) {
        dim3 block(BX, BY, 1);
        dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, 1);
        k_prolong_correct2d<T><<<grid, block, 0, st>>>(g, coarse, fine_u);
        return cudaGetLastError();
    }
    if constexpr (std::is_same<T, float>::value) {
        const bool aligned = ((reinterpret_cast<uintptr_t>(coarse) | reinterpret_cast<uintptr_t>(fine_u)) & 15) == 0;
        if ((g.nx & 3) == 0 && (g.ny & 1) == 0 && (g.nz & 1) == 0 && aligned) {
            const long long gx = (g.nx / 4 + BX - 1) / BX, gy = (g.ny / 2 + BY - 1) / BY;
            const long long chunks = std::min<long long>(g.nz / 2, std::max(1LL, 16LL * 152 / (gx * gy)));
            int kc = (int)((g.nz + chunks - 1) / chunks);
            kc += kc & 1;
            dim3 block(BX, BY, 1);
            dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)((g.nz + kc - 1) / kc));
            k_prolong_correct4<<<grid, block, 0, st>>>(g, coarse, fine_u, kc);
            return cudaGetLastError();
        }
    }
    const int kc = even_kchunk(g);
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kc - 1) / kc);
    k_prolong_correct<T><<<grid, block, 0, st>>>(g, coarse, fine_u, kc);
    return cudaGetLastError();
}

cudaError_t launch_update_residual(const LevelGeom& g, double* phi, const float* e, double* r64, float* r32,
                                  Partial* partials, int* nblocks_out, cudaStream_t st) {
    const bool uniform4 = g.ihx2 == g.ihy2 && g.ihy2 == g.ihz2;
    const bool aligned = ((reinterpret_cast<uintptr_t>(phi) | reinterpret_cast<uintptr_t>(e) |
                           reinterpret_cast<uintptr_t>(r64) | reinterpret_cast<uintptr_t>(r32)) & 15) == 0;
    if ((g.nx & 3) == 0 && aligned) {
        // as many blocks as the scalar residual launch at most (the partials buffer)
        const long long gx = (g.nx / 4 + BX - 1) / BX, gy = (g.ny + BY - 1) / BY;
        const long long chunks = std::min<long long>(g.nz, std::max(1LL, residual_blocks(g) / (gx * gy)));
        const int kc = (int)((g.nz + chunks - 1) / chunks);
        dim3 block(BX, BY, 1);
        dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)((g.nz + kc - 1) / kc));
        if (uniform4) k_update_residual4<true><<<grid, block, 0, st>>>(g, phi, e, r64, r32, partials, kc);
        else k_update_residual4<false><<<grid, block, 0, st>>>(g, phi, e, r64, r32, partials, kc);
        if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
        return cudaGetLastError();
    }
    const int kc = kchunk_for(g, BX, BY);
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kc - 1) / kc);
    const bool uniform = g.ihx2 == g.ihy2 && g.ihy2 == g.ihz2;
    if (uniform) k_update_residual<true><<<grid, block, 0, st>>>(g, phi, e, r64, r32, partials, kc);
    else k_update_residual<false><<<grid, block, 0, st>>>(g, phi, e, r64, r32, partials, kc);
    if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
    return cudaGetLastError();
}

cudaError_t launch_residual_exact(const LevelGeom& g, const double* u, const double* rhs, float* r_out,
                                  double* r_full, Partial* partials, unsigned* scratch, int* nblocks_out,
                                  int* nkernels, cudaStream_t st) {
    const bool aligned = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(rhs) |
                           reinterpret_cast<uintptr_t>(r_out) | reinterpret_cast<uintptr_t>(r_full)) & 15) == 0;
    if ((g.nx & 3) != 0 || !aligned || !r_out || !r_full || !scratch) {
        if (nkernels) *nkernels = 1;
        return launch_residual<double, float>(g, u, rhs, r_out, partials, nblocks_out, st, r_full);
    }
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const long long n = (long long)g.nx * g.ny * g.nz;
    k_max_exponent<<<(unsigned)std::min<long long>(kSumBlocks, (n / 2 + 255) / 256 + 1), 256, 0, st>>>(g, u, n,
                                                                                                      scratch);
    // as many blocks as the scalar residual launch at most (the partials buffer)
    const long long gx = (g.nx / 4 + BX - 1) / BX, gy = (g.ny + BY - 1) / BY;
    const long long chunks = std::min<long long>(g.nz, std::max(1LL, residual_blocks(g) / (gx * gy)));
    const int kc = (int)((g.nz + chunks - 1) / chunks);
    dim3 block(BX, BY, 1);
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)((g.nz + kc - 1) / kc));
    const bool uniform = g.ihx2 == g.ihy2 && g.ihy2 == g.ihz2;
    const bool faces = has_faces(g);
    auto run = [&](auto kernel) -> cudaError_t {
        const cudaError_t ea = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)sizeof(FxSmem));
        if (ea != cudaSuccess) return ea;
        kernel<<<grid, block, sizeof(FxSmem), st>>>(g, u, rhs, r_out, r_full, partials, kc, scratch);
        return cudaSuccess;
    };
    if (uniform && faces) e = run(k_residual_fx4<true, true>);
    else if (uniform) e = run(k_residual_fx4<true, false>);
    else if (faces) e = run(k_residual_fx4<false, true>);
    else e = run(k_residual_fx4<false, false>);
    if (e != cudaSuccess) return e;
    if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
    if (nkernels) *nkernels = 2;
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Partial* partials, int n, Reduced* out, cudaStream_t st) {
    k_finalize<<<1, kRedThreads, 0, st>>>(partials, n, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_subtract_mean(T* x, long long n, const Reduced* red, cudaStream_t st) {
    k_subtract_mean<T><<<grid1d(n), 256, 0, st>>>(x, n, red);
    return cudaGetLastError();
}

cudaError_t launch_scale_copy(const double* src, double* dst, double scale, long long n,
                              cudaStream_t st) {
    k_scale_copy<<<grid1d(n), 256, 0, st>>>(src, dst, scale, n);
    return cudaGetLastError();
}

cudaError_t launch_link_copy(const double* src, double* dst, double scale, bool scaled, long long n,
                             cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const bool wide = (n % 2) == 0 && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    if (!wide) return launch_scale_copy(src, dst, scaled ? scale : 1.0, n, st);
    const long long n2 = n / 2;
    const long long b = std::min<long long>((n2 + 1023) / 1024, 2048);
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
    if (scaled)
        k_link_copy<true><<<(unsigned)b, 256, 0, st>>>(s2, d2, scale, n2);
    else
        k_link_copy<false><<<(unsigned)b, 256, 0, st>>>(s2, d2, 1.0, n2);
    return cudaGetLastError();
}

cudaError_t launch_add_f32_to_f64(double* phi, const float* e, long long n, cudaStream_t st) {
    k_add_f32_to_f64<<<grid1d(n), 256, 0, st>>>(phi, e, n);
    return cudaGetLastError();
}

cudaError_t launch_sub_mean_f64(double* x, long long n, const Reduced* red, cudaStream_t st) {
    return launch_subtract_mean<double>(x, n, red, st);
}

cudaError_t launch_sum_partials_f64(const double* x, long long n, Partial* partials,
                                    int* nblocks_out, cudaStream_t st) {
    const int nb = grid1d(n);
    k_sum_f64<<<nb, 256, 0, st>>>(x, n, partials);
    if (nblocks_out) *nblocks_out = nb;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gsrb(const LevelGeom& g, int colour, double omega, T* u, const T* rhs, cudaStream_t st) {
    const int kc = kchunk_for(g, BX, BY);
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kc - 1) / kc);
    if (has_faces(g)) k_gsrb<T, true><<<grid, block, 0, st>>>(g, colour & 1, T(omega), u, rhs, kc);
    else k_gsrb<T, false><<<grid, block, 0, st>>>(g, colour & 1, T(omega), u, rhs, kc);
    return cudaGetLastError();
}

cudaError_t launch_gravity(const LevelGeom& g, const double* phi, double* out, const double c[3], unsigned* scratch,
                           int* nkernels, cudaStream_t st) {
    const int kc = kchunk_for(g, BX, BY);
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kc - 1) / kc);
    const unsigned* mexp = nullptr;
    if (scratch && (reinterpret_cast<uintptr_t>(phi) & 15) == 0) {
        // the exact fixed-point differences on the level's scale
        cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        const long long n = (long long)g.nx * g.ny * g.nz;
        k_max_exponent<<<(unsigned)std::min<long long>(kSumBlocks, (n / 2 + 255) / 256 + 1), 256, 0, st>>>(g, phi, n,
                                                                                                          scratch);
        mexp = scratch;
    }
    if (mexp && (g.nx & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        // 4-cell strips, planes staged in shared memory: about three waves of
        // two CTAs per SM, whole z chunks
        const long long gx = (g.nx / 4 + BX - 1) / BX, gy = (g.ny + BY - 1) / BY;
        const long long want = 6 * sm_count();
        const long long chunks = std::min<long long>(g.nz, std::max(1LL, (want + gx * gy - 1) / (gx * gy)));
        const int kz = (int)((g.nz + chunks - 1) / chunks);
        dim3 sgrid((unsigned)gx, (unsigned)gy, (unsigned)((g.nz + kz - 1) / kz));
        cudaError_t e = cudaFuncSetAttribute(k_gravity_fx4, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(GvSmem));
        if (e != cudaSuccess) return e;
        k_gravity_fx4<<<sgrid, block, sizeof(GvSmem), st>>>(g, phi, out, c[0], c[1], c[2], kz, mexp);
    } else {
        k_gravity_stream<<<grid, block, 0, st>>>(g, phi, out, c[0], c[1], c[2], kc, mexp);
    }
    if (nkernels) *nkernels = mexp ? 2 : 1;
    return cudaGetLastError();
}

// Explicit instantiations.
template cudaError_t launch_gsrb<float>(const LevelGeom&, int, double, float*, const float*, cudaStream_t);
template cudaError_t launch_gsrb<double>(const LevelGeom&, int, double, double*, const double*, cudaStream_t);
template cudaError_t launch_stage<float>(const LevelGeom&, int, bool, const StageCoef&, const float*,
                                         const float*, const float*, const float*, const float*,
                                         float*, float*, cudaStream_t);
template cudaError_t launch_stage<double>(const LevelGeom&, int, bool, const StageCoef&, const double*,
                                          const double*, const double*, const double*,
                                          const double*, double*, double*, cudaStream_t);
template cudaError_t launch_residual_zero<double>(const LevelGeom&, const double*, double*, Partial*, int*,
                                                  cudaStream_t, double*, int*);
template cudaError_t launch_residual_zero<float>(const LevelGeom&, const double*, float*, Partial*, int*,
                                                 cudaStream_t, double*, int*);
template cudaError_t launch_residual<double, double>(const LevelGeom&, const double*, const double*,
                                                     double*, Partial*, int*, cudaStream_t, double*);
template cudaError_t launch_residual<double, float>(const LevelGeom&, const double*, const double*,
                                                    float*, Partial*, int*, cudaStream_t, double*);
template cudaError_t launch_residual<float, float>(const LevelGeom&, const float*, const float*,
                                                   float*, Partial*, int*, cudaStream_t, float*);
template cudaError_t launch_residual_restrict<float>(const LevelGeom&, const float*, const float*,
                                                     float*, Partial*, int*, cudaStream_t);
template cudaError_t launch_residual_restrict<double>(const LevelGeom&, const double*, const double*,
                                                      double*, Partial*, int*, cudaStream_t);
template cudaError_t launch_prolong_correct<float>(const LevelGeom&, const float*, float*, cudaStream_t);
template cudaError_t launch_prolong_correct<double>(const LevelGeom&, const double*, double*,
                                                    cudaStream_t);
template cudaError_t launch_subtract_mean<float>(float*, long long, const Reduced*, cudaStream_t);
template cudaError_t launch_subtract_mean<double>(double*, long long, const Reduced*, cudaStream_t);

}  // namespace sg
