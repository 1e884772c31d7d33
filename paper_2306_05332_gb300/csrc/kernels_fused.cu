// Fused RKL super-step: all s stages of one super-step (App. A, Eq.
// RKL_intermediate_source) in one pass over HBM (temporal blocking).
//
// A CTA owns a TX x TY column of the level and streams it along z.  The tile
// is widened by a halo (s cells in y; HX >= s cells in x, a multiple of 4 so
// that shared-memory rows and global strips stay 16-byte aligned); stage j is
// computed on the tile widened by s - j cells, so after s stages the tile
// itself is exact.  Work is done in strips of four consecutive x cells, read
// and written as float4.
//
// Pipeline.  In phase t of the stream, stage j works on plane t - (2j - 1).
// Lagging each stage two planes behind the previous one means every stage
// reads only planes finished in an earlier phase, so the stages of a phase are
// independent and one __syncthreads() per phase suffices.  Every stage output,
// Y0, f and Z0 = tau (L Y0 - f) live in rings of z-planes in shared memory;
// Y0 and f planes arrive by cp.async one phase ahead.
//
// HBM traffic per super-step: read Y0 + read f + write Y_s (12 B/cell FP32;
// 8 B/cell when Y0 = 0) instead of 12-24 B/cell per stage.  Halo cells are
// re-read from L2 by neighbouring tiles, which stream the same planes.
//
// Boundaries (the error equation of the FP32 V-cycle has no Dirichlet data):
//   Dirichlet (Eq. error_ghost): the ghost is -centre, applied inline at the
//     wall; halo cells outside the box are computed from stale shared memory
//     but never read by a cell inside the box, and never written to HBM.
//   periodic (Eq. periodic): loads wrap around, so the halo holds the periodic
//     image and halo cells are computed like interior ones.
// The output must not alias Y0 (a neighbouring tile may still read Y0's halo).
#include "sg_internal.cuh"

#include <algorithm>
#include <type_traits>

namespace sg {

namespace {

constexpr int FT_X = 32;
constexpr int FT_THREADS = 512;

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ int wrap(int v, int n) {
    int m = v % n;
    return m < 0 ? m + n : m;
}

template <int R>
__device__ __forceinline__ int slot(int p) {
    const int m = p % R;
    return m < 0 ? m + R : m;
}

template <int S, int ORDER, bool ZERO>
struct FusedCfg {
    static constexpr int TX = FT_X;
    static constexpr int TY = S <= 3 ? 16 : (S <= 5 ? 8 : 4);
    static constexpr int HX = S <= 4 ? 4 : 8;                                  // x halo (multiple of 4)
    static constexpr int W = TX + 2 * HX;                                      // plane row, floats
    static constexpr int H = TY + 2 * S;                                       // plane rows
    static constexpr int Q = W / 4;                                            // float4 strips per row
    static constexpr int P = W * H;                                            // floats per plane
    // ring depths (planes) for stage j on plane t - (2j - 1), loads one phase ahead
    static constexpr int R0 = ZERO ? 1 : (ORDER == 2 ? 2 * S + 1 : 5);         // Y0
    static constexpr int RF = 2 * S + 1;                                       // f
    static constexpr int RZ = (ORDER == 2 && !ZERO) ? 2 * S - 1 : 1;           // Z0
    static constexpr int RY = 5;                                               // each Y_j, j < s
    static constexpr int NPLANES = (ZERO ? 0 : R0) + RF + ((ORDER == 2 && !ZERO) ? RZ : 0) + RY * (S - 1);
    static constexpr size_t BYTES = size_t(NPLANES) * P * sizeof(float);
    static_assert(BYTES <= 227u * 1024u, "fused super-step rings exceed the shared memory of one CTA");
    // strips of stage j: x cells [HX - (S - j), HX + TX + (S - j)) rounded out to strips
    __host__ __device__ static constexpr int qlo(int j) { return (HX - (S - j)) / 4; }
    __host__ __device__ static constexpr int qhi(int j) { return (HX + TX + (S - j) + 3) / 4; }
};

template <int R>
__device__ __forceinline__ int back(int s, int k) {     // slot of plane t - k, given s = slot of t
    const int v = s - (k % R);
    return v < 0 ? v + R : v;
}

template <int S, int ORDER, bool ZERO, bool UNIF, bool V16>
__global__ void __launch_bounds__(FT_THREADS)
k_superstep_fused(const __grid_constant__ LevelGeom g, const __grid_constant__ FusedCoef cf,
                  const float* __restrict__ y0g, const float* __restrict__ fg, float* __restrict__ outg,
                  int kchunk) {
    using C = FusedCfg<S, ORDER, ZERO>;
    constexpr int W = C::W, H = C::H, P = C::P, Q = C::Q;
    constexpr int R0 = C::R0, RF = C::RF, RZ = C::RZ, RY = C::RY;
    static_assert(H * Q <= FT_THREADS, "one load strip per thread");
    extern __shared__ __align__(16) float sm[];
    float* const sY0 = sm;
    float* const sF = sY0 + (ZERO ? 0 : R0) * P;
    float* const sZ = sF + RF * P;
    float* const sY = sZ + ((ORDER == 2 && !ZERO) ? RZ : 0) * P;
    const int tid = threadIdx.x;
    const int X0 = blockIdx.x * C::TX - C::HX;      // global x / y of local (0, 0)
    const int Y0 = blockIdx.y * C::TY - S;
    const int nx = g.nx, ny = g.ny, nz = g.nz, plane = g.nx * g.ny;
    const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
    const float ihx2 = g.ihx2f, ihy2 = g.ihy2f, ihz2 = g.ihz2f;

    // ---- this thread's strip in every stage and in the plane loads (fixed for the whole stream)
    int so[S + 1], sgx[S + 1], sgy[S + 1];
    unsigned on = 0u;
#pragma unroll
    for (int j = 1; j <= S; ++j) {
        const int nq = C::qhi(j) - C::qlo(j), nr = H - 2 * j;
        so[j] = 0;
        sgx[j] = 0;
        sgy[j] = 0;
        if (tid < nr * nq) {
            const int r = j + tid / nq, q = C::qlo(j) + tid % nq;
            const int gy = Y0 + r;
            if (py || (gy >= 0 && gy < ny)) {
                on |= 1u << j;
                so[j] = r * W + 4 * q;
                sgx[j] = X0 + 4 * q;
                sgy[j] = gy;
            }
        }
    }
    int ld_d = 0, ld_g = -1;                        // destination in a plane; in-plane source (V16)
    int ld_ge[4] = {-1, -1, -1, -1};                // per-cell sources (scalar copies)
    if (tid < H * Q) {
        const int r = tid / Q, q = tid % Q;
        ld_d = r * W + 4 * q;
        int gy = Y0 + r;
        const bool rowok = (gy >= 0 && gy < ny) || py;
        if (rowok) {
            gy = wrap(gy, ny);
            const int gx0 = X0 + 4 * q;
            if constexpr (V16) {
                if ((gx0 >= 0 && gx0 < nx) || px) ld_g = gy * nx + wrap(gx0, nx);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int gx = gx0 + e;
                    if ((gx >= 0 && gx < nx) || px) ld_ge[e] = gy * nx + wrap(gx, nx);
                }
            }
        }
    }
    auto load = [&](float* dst, const float* src, int p) {
        const float* b = src + (long long)(pz ? wrap(p, nz) : p) * plane;
        if constexpr (V16) {
            if (ld_g >= 0) cp_async16(dst + ld_d, b + ld_g);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (ld_ge[e] >= 0) cp_async4(dst + ld_d + e, b + ld_ge[e]);
        }
    };

    // ---- one strip of stage J on plane p; s*: ring slots of plane t
    auto stage = [&](auto JJ, int p, int s0, int sf, int sz, int sy) {
        constexpr int J = decltype(JJ)::value;
        if (!(on & (1u << J))) return;
        constexpr int L = 2 * J - 1;                // lag: p = t - L
        const int o = so[J], gx0 = sgx[J], gy = sgy[J];
        const float* yc;
        const float* ym;
        const float* yq;
        if constexpr (J == 1) {
            yc = sY0 + back<R0>(s0, L) * P;
            ym = sY0 + back<R0>(s0, L + 1) * P;
            yq = sY0 + back<R0>(s0, L - 1) * P;
        } else {
            const float* b = sY + (J - 2) * RY * P;
            yc = b + back<RY>(sy, L) * P;
            ym = b + back<RY>(sy, L + 1) * P;
            yq = b + back<RY>(sy, L - 1) * P;
        }
        const float4 f4 = *reinterpret_cast<const float4*>(sF + back<RF>(sf, L) * P + o);
        const float fv[4] = {f4.x, f4.y, f4.z, f4.w};
        float v[4];
        if constexpr (J == 1 && ZERO) {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = cf.mut1 * (cf.tau * (0.0f - fv[e]));   // Y0 = 0
        } else {
            const float4 c4 = *reinterpret_cast<const float4*>(yc + o);
            const float4 n4 = *reinterpret_cast<const float4*>(yc + o - W);
            const float4 s4 = *reinterpret_cast<const float4*>(yc + o + W);
            const float4 d4 = *reinterpret_cast<const float4*>(ym + o);
            const float4 u4 = *reinterpret_cast<const float4*>(yq + o);
            const float left = yc[o - 1], right = yc[o + 4];
            const float cc[4] = {c4.x, c4.y, c4.z, c4.w};
            const float yn[4] = {n4.x, n4.y, n4.z, n4.w};
            const float ys[4] = {s4.x, s4.y, s4.z, s4.w};
            const float zd[4] = {d4.x, d4.y, d4.z, d4.w};
            const float zu[4] = {u4.x, u4.y, u4.z, u4.w};
            const bool ylo = !py && gy == 0, yhi = !py && gy == ny - 1;
            const bool zlo = !pz && p == 0, zhi = !pz && p == nz - 1;
            float y2[4] = {0.f, 0.f, 0.f, 0.f}, y0x[4] = {0.f, 0.f, 0.f, 0.f}, z0x[4] = {0.f, 0.f, 0.f, 0.f};
            if constexpr (J >= 2 && !(J == 2 && ZERO)) {
                const float* a = (J >= 3) ? sY + ((J - 3) * RY + back<RY>(sy, L)) * P : sY0 + back<R0>(s0, L) * P;
                const float4 a4 = *reinterpret_cast<const float4*>(a + o);
                y2[0] = a4.x; y2[1] = a4.y; y2[2] = a4.z; y2[3] = a4.w;
            }
            if constexpr (J >= 2 && ORDER == 2 && !ZERO) {
                const float4 b4 = *reinterpret_cast<const float4*>(sY0 + back<R0>(s0, L) * P + o);
                const float4 z4 = *reinterpret_cast<const float4*>(sZ + back<RZ>(sz, L) * P + o);
                y0x[0] = b4.x; y0x[1] = b4.y; y0x[2] = b4.z; y0x[3] = b4.w;
                z0x[0] = z4.x; z0x[1] = z4.y; z0x[2] = z4.z; z0x[3] = z4.w;
            }
            float zout[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float ce = cc[e];
                float xm = e == 0 ? left : cc[e - 1];
                float xp = e == 3 ? right : cc[e + 1];
                if (!px && gx0 + e == 0) xm = -ce;
                if (!px && gx0 + e == nx - 1) xp = -ce;
                const float ymv = ylo ? -ce : yn[e];
                const float ypv = yhi ? -ce : ys[e];
                const float zmv = zlo ? -ce : zd[e];
                const float zpv = zhi ? -ce : zu[e];
                float Lf;
                if constexpr (UNIF) {
                    Lf = fmaf(((xm + xp) + (ymv + ypv)) + (zmv + zpv) - 6.0f * ce, ihx2, -fv[e]);
                } else {
                    const float two_c = 2.0f * ce;
                    Lf = (((xm - two_c) + xp) * ihx2 + ((ymv - two_c) + ypv) * ihy2 +
                          ((zmv - two_c) + zpv) * ihz2) - fv[e];
                }
                if constexpr (J == 1) {
                    const float z = cf.tau * Lf;
                    zout[e] = z;
                    v[e] = ce + cf.mut1 * z;
                } else {
                    float ve = cf.mu[J] * ce + cf.nu[J] * y2[e] + cf.mut_tau[J] * Lf;
                    if constexpr (ORDER == 2) {
                        const float z0v = ZERO ? cf.tau * (0.0f - fv[e]) : z0x[e];
                        ve = ve + cf.c0[J] * y0x[e] + cf.gt[J] * z0v;
                    }
                    v[e] = ve;
                }
            }
            if constexpr (J == 1 && ORDER == 2 && !ZERO)
                *reinterpret_cast<float4*>(sZ + back<RZ>(sz, L) * P + o) =
                    make_float4(zout[0], zout[1], zout[2], zout[3]);
        }
        if constexpr (J == S) {
            if (gy >= ny) return;                   // ragged tile edge (periodic y)
            const long long ob = (long long)p * plane + (long long)gy * nx;
            if (V16 && gx0 + 3 < nx) {
                *reinterpret_cast<float4*>(outg + ob + gx0) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (gx0 + e < nx) outg[ob + gx0 + e] = v[e];
            }
        } else {
            *reinterpret_cast<float4*>(sY + ((J - 1) * RY + back<RY>(sy, L)) * P + o) =
                make_float4(v[0], v[1], v[2], v[3]);
        }
    };

    const int kz0 = blockIdx.z * kchunk;
    const int kz1 = min(kz0 + kchunk, nz);
    int lo_load = kz0 - S, hi_load = kz1 + S;       // planes of Y0 / f to stage: [lo, hi)
    if (!pz) {
        lo_load = max(lo_load, 0);
        hi_load = min(hi_load, nz);
    }
    for (int p = lo_load; p < min(lo_load + 2, hi_load); ++p) {
        if constexpr (!ZERO) load(sY0 + slot<R0>(p) * P, y0g, p);
        load(sF + slot<RF>(p) * P, fg, p);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    // stage j's planes are [kz0 - (s - j), kz1 + (s - j)), clipped to the box for Dirichlet z
    auto in_range = [&](int j, int p) {
        int lo = kz0 - (S - j), hi = kz1 + (S - j);
        if (!pz) {
            lo = max(lo, 0);
            hi = min(hi, nz);
        }
        return p >= lo && p < hi;
    };
    const int t_first = lo_load + 1;
    const int t_end = kz1 - 1 + (2 * S - 1);
    int s0 = slot<R0>(t_first), sf = slot<RF>(t_first), sz = slot<RZ>(t_first), sy = slot<RY>(t_first);
    for (int t = t_first; t <= t_end; ++t) {
        if (t + 1 < hi_load) {
            const int n0 = s0 + 1 == R0 ? 0 : s0 + 1, nf = sf + 1 == RF ? 0 : sf + 1;
            if constexpr (!ZERO) load(sY0 + n0 * P, y0g, t + 1);
            load(sF + nf * P, fg, t + 1);
        }
        cp_async_commit();
        if (in_range(1, t - 1)) stage(std::integral_constant<int, 1>{}, t - 1, s0, sf, sz, sy);
        if constexpr (S >= 2) if (in_range(2, t - 3)) stage(std::integral_constant<int, 2>{}, t - 3, s0, sf, sz, sy);
        if constexpr (S >= 3) if (in_range(3, t - 5)) stage(std::integral_constant<int, 3>{}, t - 5, s0, sf, sz, sy);
        if constexpr (S >= 4) if (in_range(4, t - 7)) stage(std::integral_constant<int, 4>{}, t - 7, s0, sf, sz, sy);
        if constexpr (S >= 5) if (in_range(5, t - 9)) stage(std::integral_constant<int, 5>{}, t - 9, s0, sf, sz, sy);
        if constexpr (S >= 6) if (in_range(6, t - 11)) stage(std::integral_constant<int, 6>{}, t - 11, s0, sf, sz, sy);
        cp_async_wait_all();
        __syncthreads();
        s0 = s0 + 1 == R0 ? 0 : s0 + 1;
        sf = sf + 1 == RF ? 0 : sf + 1;
        sz = sz + 1 == RZ ? 0 : sz + 1;
        sy = sy + 1 == RY ? 0 : sy + 1;
    }
}

int g_num_sms = 152;

template <int S, int ORDER, bool ZERO, bool UNIF, bool V16>
struct Resident {
    static int per_sm;      // CTAs of this instantiation resident per SM (set at configure time)
};
template <int S, int ORDER, bool ZERO, bool UNIF, bool V16>
int Resident<S, ORDER, ZERO, UNIF, V16>::per_sm = 1;

template <int S, int ORDER, bool ZERO, bool UNIF, bool V16>
cudaError_t launch_one(const LevelGeom& g, const FusedCoef& cf, const float* y0, const float* f, float* out,
                       cudaStream_t st) {
    using C = FusedCfg<S, ORDER, ZERO>;
    const long long gx = (g.nx + C::TX - 1) / C::TX, gy = (g.ny + C::TY - 1) / C::TY;
    // Split z so that all CTAs are resident in one wave (no partial second wave);
    // a chunk re-stages 2s halo planes and its pipeline fills over 2s phases,
    // so chunks stay at least 4s planes long.
    const long long slots = (long long)g_num_sms * Resident<S, ORDER, ZERO, UNIF, V16>::per_sm;
    long long chunks = std::max(1LL, slots / (gx * gy));
    chunks = std::min<long long>(chunks, std::max(1, g.nz / (4 * S)));
    const int kchunk = (int)((g.nz + chunks - 1) / chunks);
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)((g.nz + kchunk - 1) / kchunk));
    k_superstep_fused<S, ORDER, ZERO, UNIF, V16><<<grid, FT_THREADS, C::BYTES, st>>>(g, cf, y0, f, out, kchunk);
    return cudaGetLastError();
}

template <int S, int ORDER, bool ZERO, bool UNIF, bool V16>
cudaError_t configure_one() {
    using C = FusedCfg<S, ORDER, ZERO>;
    auto k = k_superstep_fused<S, ORDER, ZERO, UNIF, V16>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, FT_THREADS, C::BYTES);
    if (e != cudaSuccess) return e;
    Resident<S, ORDER, ZERO, UNIF, V16>::per_sm = n > 0 ? n : 1;
    return cudaSuccess;
}

template <int S, int ORDER, bool ZERO>
cudaError_t launch_uv(bool unif, bool v16, const LevelGeom& g, const FusedCoef& cf, const float* y0,
                      const float* f, float* out, cudaStream_t st) {
    if (unif) return v16 ? launch_one<S, ORDER, ZERO, true, true>(g, cf, y0, f, out, st)
                         : launch_one<S, ORDER, ZERO, true, false>(g, cf, y0, f, out, st);
    return v16 ? launch_one<S, ORDER, ZERO, false, true>(g, cf, y0, f, out, st)
               : launch_one<S, ORDER, ZERO, false, false>(g, cf, y0, f, out, st);
}

template <int S>
cudaError_t dispatch(int order, bool zero, const LevelGeom& g, const FusedCoef& cf, const float* y0,
                     const float* f, float* out, cudaStream_t st) {
    const bool unif = g.ihx2f == g.ihy2f && g.ihy2f == g.ihz2f;
    const bool v16 = (g.nx & 3) == 0;
    if (order == 1) return zero ? launch_uv<S, 1, true>(unif, v16, g, cf, y0, f, out, st)
                                : launch_uv<S, 1, false>(unif, v16, g, cf, y0, f, out, st);
    return zero ? launch_uv<S, 2, true>(unif, v16, g, cf, y0, f, out, st)
                : launch_uv<S, 2, false>(unif, v16, g, cf, y0, f, out, st);
}

template <int S, int ORDER, bool ZERO>
cudaError_t configure_ouv() {
    cudaError_t e;
    if ((e = configure_one<S, ORDER, ZERO, true, true>()) != cudaSuccess) return e;
    if ((e = configure_one<S, ORDER, ZERO, true, false>()) != cudaSuccess) return e;
    if ((e = configure_one<S, ORDER, ZERO, false, true>()) != cudaSuccess) return e;
    return configure_one<S, ORDER, ZERO, false, false>();
}

template <int S>
cudaError_t configure_s() {
    cudaError_t e;
    if ((e = configure_ouv<S, 1, true>()) != cudaSuccess) return e;
    if ((e = configure_ouv<S, 1, false>()) != cudaSuccess) return e;
    if ((e = configure_ouv<S, 2, true>()) != cudaSuccess) return e;
    return configure_ouv<S, 2, false>();
}

}  // namespace

bool fused_supported(int order, int s) { return (order == 1 || order == 2) && s >= 2 && s <= kFusedMaxS; }

cudaError_t fused_configure() {
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = lean_configure()) != cudaSuccess) return e;       // s = 2, 3 (kernels_superstep.cu)
    if ((e = configure_s<4>()) != cudaSuccess) return e;
    if ((e = configure_s<5>()) != cudaSuccess) return e;
    return configure_s<6>();
}

cudaError_t launch_superstep_fused(const LevelGeom& g, int order, int s, bool zero_y0, const FusedCoef& cf,
                                   const float* y0, const float* f, float* out, cudaStream_t st, int tile_rows,
                                   bool tma) {
    switch (s) {
        case 2:
        case 3: return launch_superstep_lean(g, order, s, zero_y0, cf, y0, f, out, st, tile_rows, tma);
        case 4: return dispatch<4>(order, zero_y0, g, cf, y0, f, out, st);
        case 5: return dispatch<5>(order, zero_y0, g, cf, y0, f, out, st);
        case 6: return dispatch<6>(order, zero_y0, g, cf, y0, f, out, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sg
