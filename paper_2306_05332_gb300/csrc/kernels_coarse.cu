// Coarsest-level solver: the whole level lives in one CTA's shared memory and
// the accelerated RKL1 iteration of App. A.5 runs there with __syncthreads()
// between stages, so a coarse solve of hundreds of stages is one launch.
//
// Stage k of super-step s (App. A, Eq. RKL_intermediate_source, first order):
//   Y1 = Y0 + tau_unit (L Y0 - f)
//   Yj = mu_j Y_{j-1} + nu_j Y_{j-2} + mu_j tau_unit (L Y_{j-1} - f)
// with mu_j = (2j-1)/j, nu_j = (1-j)/j and tau_unit = w1 tau = tau_frac * 2 / lambda_max
// (since tau_max w1 = dt_par = 2 / lambda_max).  Before every super-step the
// relative residual is compared with `tol` (0 = run exactly max_ss super-steps).
// Boundaries: homogeneous Dirichlet (Eq. error_ghost) or periodic.
#include "sg_internal.cuh"

#include <cstdint>
#include <type_traits>

namespace sg {

namespace {

constexpr int kCoarseThreads = 1024;
constexpr size_t kSmemLimit = 227u * 1024u - 1024u;

template <typename T>
__device__ __forceinline__ T lap_smem(const T* u, int nx, int ny, int nz, const int* per, T ihx2,
                                      T ihy2, T ihz2, int i, int j, int k) {
    const int sy = nx, sz = nx * ny;
    const int t = k * sz + j * sy + i;
    const T c = u[t];
    const T xm = i > 0 ? u[t - 1] : (per[0] ? u[t + nx - 1] : -c);
    const T xp = i < nx - 1 ? u[t + 1] : (per[0] ? u[t - (nx - 1)] : -c);
    const T ym = j > 0 ? u[t - sy] : (per[1] ? u[t + (ny - 1) * sy] : -c);
    const T yp = j < ny - 1 ? u[t + sy] : (per[1] ? u[t - (ny - 1) * sy] : -c);
    const T zm = k > 0 ? u[t - sz] : (per[2] ? u[t + (nz - 1) * sz] : -c);
    const T zp = k < nz - 1 ? u[t + sz] : (per[2] ? u[t - (nz - 1) * sz] : -c);
    const T two_c = T(2) * c;
    return ((xm - two_c) + xp) * ihx2 + ((ym - two_c) + yp) * ihy2 + ((zm - two_c) + zp) * ihz2;
}

template <typename T>
__device__ T block_sum(T v, T* scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? scratch[lane] : T(0);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) scratch[32] = v;
    }
    __syncthreads();
    const T r = scratch[32];
    __syncthreads();
    return r;
}

// At most kMaxCells cells per thread: the level fits shared memory, so
// n <= kSmemLimit / (4 sizeof(float)) < kMaxCells * kCoarseThreads.
constexpr int kMaxCells = 16;

template <typename T, int MAXC>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_solve(const CoarseParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[33];
    const int nx = p.g.nx, ny = p.g.ny, nz = p.g.nz;
    const int n = nx * ny * nz;
    T* f = reinterpret_cast<T*>(smem_raw);
    T* buf[3] = {f + n, f + 2 * n, f + 3 * n};
    const T* rhs = static_cast<const T*>(p.rhs);
    const T ihx2 = ih2x<T>(p.g), ihy2 = ih2y<T>(p.g), ihz2 = ih2z<T>(p.g);
    int per[3] = {p.g.per[0], p.g.per[1], p.g.per[2]};

    // this thread's cells t = tid + m * blockDim, coordinates packed once
    int cell[MAXC];
#pragma unroll
    for (int m = 0; m < MAXC; ++m) {
        const int t = threadIdx.x + m * blockDim.x;
        cell[m] = t < n ? ((t % nx) | (((t / nx) % ny) << 10) | ((t / (nx * ny)) << 20)) : -1;
    }
    auto lap = [&](const T* y, int c) {
        return lap_smem(y, nx, ny, nz, per, ihx2, ihy2, ihz2, c & 1023, (c >> 10) & 1023, c >> 20);
    };

    T local = T(0);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const T v = rhs[t];
        f[t] = v;
        buf[0][t] = T(0);
        local += v * v;
    }
    __syncthreads();
    const T r0sq = block_sum(local, red);         // ||f - L 0||^2 with homogeneous ghosts
    const T tol = T(p.tol);                       // converted once; kept in a register
    const T tau_unit_t = T(p.tau_unit);
    const T tolsq = tol * tol * r0sq;

    int cur = 0;
    int done = 0;
    for (int ss = 0; ss < p.max_ss; ++ss) {
        if (tol > T(0)) {
            T acc = T(0);
#pragma unroll
            for (int m = 0; m < MAXC; ++m) {
                if (cell[m] < 0) break;
                const int t = threadIdx.x + m * blockDim.x;
                const T r = f[t] - lap(buf[cur], cell[m]);
                acc += r * r;
            }
            const T rsq = block_sum(acc, red);
            if (rsq <= tolsq) break;
        }
        const int s = p.sched[ss];
        int prev = -1;
        for (int jst = 1; jst <= s; ++jst) {
            const int nxt = (cur + 1) % 3 == prev ? (cur + 2) % 3 : (cur + 1) % 3;
            // coefficients in the kernel's precision (FP64 issue is 1/64 of FP32 on GB300)
            const T mu = (T(2) * T(jst) - T(1)) / T(jst);
            const T nu = (T(1) - T(jst)) / T(jst);
            const T tu = tau_unit_t;
            const T mut = mu * tu;
            const T* yc = buf[cur];
            const T* yp = prev >= 0 ? buf[prev] : buf[cur];
            T* yn = buf[nxt];
#pragma unroll
            for (int m = 0; m < MAXC; ++m) {
                if (cell[m] < 0) break;
                const int t = threadIdx.x + m * blockDim.x;
                const T Lf = lap(yc, cell[m]) - f[t];
                if (jst == 1) yn[t] = yc[t] + tu * Lf;
                else yn[t] = mu * yc[t] + nu * yp[t] + mut * Lf;
            }
            __syncthreads();
            prev = cur;
            cur = nxt;
        }
        ++done;
    }
    T* out = static_cast<T*>(p.u_out);
    for (int t = threadIdx.x; t < n; t += blockDim.x) out[t] = buf[cur][t];
    if (threadIdx.x == 0 && p.ss_done) *p.ss_done = done;
}

// Levels of at most kSmallCells cells: every buffer carries a one-cell ghost
// layer, (nx+2)(ny+2)(nz+2), so the stencil reads fixed offsets with no
// boundary test.  The thread that writes a boundary cell also writes the
// ghost that mirrors it (-v across a Dirichlet wall, Eq. error_ghost; v on the
// opposite side of a periodic axis, Eq. periodic), so each ghost has one
// writer and a stage needs one barrier.  Each thread keeps its cells' padded
// indices, face flags and right-hand side in registers.
constexpr int kSmallCells = 4 * kCoarseThreads;

template <typename T>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_small(const CoarseParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[33];
    const int nx = p.g.nx, ny = p.g.ny, nz = p.g.nz;
    const int n = nx * ny * nz;
    const int px = nx + 2, pxy = px * (ny + 2), np = pxy * (nz + 2);
    T* const b0 = reinterpret_cast<T*>(smem_raw);
    const T ihx2 = ih2x<T>(p.g), ihy2 = ih2y<T>(p.g), ihz2 = ih2z<T>(p.g);
    const T diag = T(2) * (ihx2 + ihy2 + ihz2);
    const bool perx = p.g.per[0] != 0, pery = p.g.per[1] != 0, perz = p.g.per[2] != 0;
    const T* rhs = static_cast<const T*>(p.rhs);

    // this thread's cells t = tid + m * blockDim: padded index, face flags, f
    int pc[4];
    unsigned faces = 0u;                  // 6 bits per cell: -x +x -y +y -z +z
    T fv[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int t = threadIdx.x + m * blockDim.x;
        pc[m] = -1;
        fv[m] = T(0);
        if (t < n) {
            const int i = t % nx, j = (t / nx) % ny, k = t / (nx * ny);
            pc[m] = (k + 1) * pxy + (j + 1) * px + (i + 1);
            const unsigned fl = (i == 0 ? 1u : 0u) | (i == nx - 1 ? 2u : 0u) | (j == 0 ? 4u : 0u) |
                                (j == ny - 1 ? 8u : 0u) | (k == 0 ? 16u : 0u) | (k == nz - 1 ? 32u : 0u);
            faces |= fl << (6 * m);
            fv[m] = rhs[t];
        }
    }
    for (int idx = threadIdx.x; idx < 3 * np; idx += blockDim.x) b0[idx] = T(0);
    __syncthreads();

    auto lap = [&](const T* y, int q) {
        return ihx2 * (y[q - 1] + y[q + 1]) + ihy2 * (y[q - px] + y[q + px]) + ihz2 * (y[q - pxy] + y[q + pxy]) -
               diag * y[q];
    };
    // store v at cell m of y and at the ghosts that mirror it
    auto put = [&](T* y, int m, T v) {
        const int q = pc[m];
        y[q] = v;
        const unsigned fl = (faces >> (6 * m)) & 63u;
        if (fl) {
            if (fl & 1u) y[perx ? q + nx : q - 1] = perx ? v : -v;
            if (fl & 2u) y[perx ? q - nx : q + 1] = perx ? v : -v;
            if (fl & 4u) y[pery ? q + ny * px : q - px] = pery ? v : -v;
            if (fl & 8u) y[pery ? q - ny * px : q + px] = pery ? v : -v;
            if (fl & 16u) y[perz ? q + nz * pxy : q - pxy] = perz ? v : -v;
            if (fl & 32u) y[perz ? q - nz * pxy : q + pxy] = perz ? v : -v;
        }
    };

    T local = T(0);
#pragma unroll
    for (int m = 0; m < 4; ++m) local += fv[m] * fv[m];
    const T r0sq = block_sum(local, red);         // ||f - L 0||^2 with homogeneous ghosts
    const T tol = T(p.tol);
    const T tu = T(p.tau_unit);
    const T tolsq = tol * tol * r0sq;

    T* y_cur = b0;                                // all zero, ghosts included
    T* y_prev = b0 + np;
    T* y_free = b0 + 2 * np;
    int done = 0;
    for (int ss = 0; ss < p.max_ss; ++ss) {
        if (tol > T(0)) {
            T acc = T(0);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (pc[m] < 0) break;
                const T r = fv[m] - lap(y_cur, pc[m]);
                acc += r * r;
            }
            const T rsq = block_sum(acc, red);
            if (rsq <= tolsq) break;
        }
        const int s = p.sched[ss];
        for (int jst = 1; jst <= s; ++jst) {
            const T mu = (T(2) * T(jst) - T(1)) / T(jst);
            const T nu = (T(1) - T(jst)) / T(jst);
            const T mut = mu * tu;
            T* const y_new = y_free;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (pc[m] < 0) break;
                const int q = pc[m];
                const T Lf = lap(y_cur, q) - fv[m];
                put(y_new, m, jst == 1 ? y_cur[q] + tu * Lf : mu * y_cur[q] + nu * y_prev[q] + mut * Lf);
            }
            __syncthreads();
            y_free = y_prev;
            y_prev = y_cur;
            y_cur = y_new;
        }
        ++done;
    }
    T* out = static_cast<T*>(p.u_out);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int t = threadIdx.x + m * blockDim.x;
        if (pc[m] >= 0) out[t] = y_cur[pc[m]];
    }
    if (threadIdx.x == 0 && p.ss_done) *p.ss_done = done;
}

// FP32 levels with nx % 4 == 0 and at most kCoarseThreads strips of four x
// cells: one strip per thread, 16-byte loads and stores.  Rows are padded to
// nx + 8 floats with the interior at offset 4 (16-byte aligned) and the x
// ghosts at offsets 3 and nx + 4; y and z ghost rows and planes as above.
__device__ __forceinline__ float4 cld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void cst4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

__global__ void __launch_bounds__(kCoarseThreads) k_coarse_strips(const CoarseParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red[33];
    const int nx = p.g.nx, ny = p.g.ny, nz = p.g.nz;
    const int nq = nx >> 2, nstrips = nq * ny * nz;
    const int rs = nx + 8, ps = rs * (ny + 2), np = ps * (nz + 2);
    float* const b0 = reinterpret_cast<float*>(smem_raw);
    const float hx = p.g.ihx2f, hy = p.g.ihy2f, hz = p.g.ihz2f;
    const float diag = 2.0f * (hx + hy + hz);
    const bool perx = p.g.per[0] != 0, pery = p.g.per[1] != 0, perz = p.g.per[2] != 0;
    const float* rhs = static_cast<const float*>(p.rhs);

    const int sidx = threadIdx.x;
    const bool mine = sidx < nstrips;
    int q = 0, j = 0, k = 0;
    if (mine) {
        q = sidx % nq;
        j = (sidx / nq) % ny;
        k = sidx / (nq * ny);
    }
    const int pc = (k + 1) * ps + (j + 1) * rs + 4 + 4 * q;     // padded index of the strip
    const int t = (k * ny + j) * nx + 4 * q;                     // unpadded index
    float4 fv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mine) fv = cld4(rhs + t);
    for (int idx = threadIdx.x; idx < 3 * np; idx += blockDim.x) b0[idx] = 0.0f;
    __syncthreads();

    auto lap = [&](const float* y) {
        const float4 c = cld4(y + pc);
        const float l = y[pc - 1], r = y[pc + 4];
        const float4 ym = cld4(y + pc - rs), yp = cld4(y + pc + rs);
        const float4 zm = cld4(y + pc - ps), zp = cld4(y + pc + ps);
        float4 o;
        o.x = hx * (l + c.y) + hy * (ym.x + yp.x) + hz * (zm.x + zp.x) - diag * c.x;
        o.y = hx * (c.x + c.z) + hy * (ym.y + yp.y) + hz * (zm.y + zp.y) - diag * c.y;
        o.z = hx * (c.y + c.w) + hy * (ym.z + yp.z) + hz * (zm.z + zp.z) - diag * c.z;
        o.w = hx * (c.z + r) + hy * (ym.w + yp.w) + hz * (zm.w + zp.w) - diag * c.w;
        return o;
    };
    // store the strip and the ghosts that mirror it (Eq. error_ghost / Eq. periodic)
    auto put = [&](float* y, float4 v) {
        cst4(y + pc, v);
        const float4 nv = make_float4(-v.x, -v.y, -v.z, -v.w);
        if (q == 0) y[perx ? pc + nx : pc - 1] = perx ? v.x : -v.x;
        if (q == nq - 1) y[perx ? pc + 3 - nx : pc + 4] = perx ? v.w : -v.w;
        if (j == 0) cst4(y + (pery ? pc + ny * rs : pc - rs), pery ? v : nv);
        if (j == ny - 1) cst4(y + (pery ? pc - ny * rs : pc + rs), pery ? v : nv);
        if (k == 0) cst4(y + (perz ? pc + nz * ps : pc - ps), perz ? v : nv);
        if (k == nz - 1) cst4(y + (perz ? pc - nz * ps : pc + ps), perz ? v : nv);
    };

    const float r0sq = block_sum(mine ? fv.x * fv.x + fv.y * fv.y + fv.z * fv.z + fv.w * fv.w : 0.0f, red);
    const float tol = float(p.tol);
    const float tu = float(p.tau_unit);
    const float tolsq = tol * tol * r0sq;

    float* y_cur = b0;
    float* y_prev = b0 + np;
    float* y_free = b0 + 2 * np;
    int done = 0;
    for (int ss = 0; ss < p.max_ss; ++ss) {
        if (tol > 0.0f) {
            float acc = 0.0f;
            if (mine) {
                const float4 L = lap(y_cur);
                const float4 r = make_float4(fv.x - L.x, fv.y - L.y, fv.z - L.z, fv.w - L.w);
                acc = r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
            }
            if (block_sum(acc, red) <= tolsq) break;
        }
        const int s = p.sched[ss];
        for (int jst = 1; jst <= s; ++jst) {
            const float inv = 1.0f / float(jst);
            const float mu = 2.0f - inv, nu = inv - 1.0f;   // (2j - 1) / j, (1 - j) / j
            const float mut = mu * tu;
            float* const y_new = y_free;
            if (mine) {
                const float4 L = lap(y_cur);
                const float4 c = cld4(y_cur + pc);
                float4 v;
                if (jst == 1) {
                    v = make_float4(c.x + tu * (L.x - fv.x), c.y + tu * (L.y - fv.y), c.z + tu * (L.z - fv.z),
                                    c.w + tu * (L.w - fv.w));
                } else {
                    const float4 pv = cld4(y_prev + pc);
                    v = make_float4(mu * c.x + nu * pv.x + mut * (L.x - fv.x), mu * c.y + nu * pv.y + mut * (L.y - fv.y),
                                    mu * c.z + nu * pv.z + mut * (L.z - fv.z), mu * c.w + nu * pv.w + mut * (L.w - fv.w));
                }
                put(y_new, v);
            }
            __syncthreads();
            y_free = y_prev;
            y_prev = y_cur;
            y_cur = y_new;
        }
        ++done;
    }
    if (mine) cst4(static_cast<float*>(p.u_out) + t, cld4(y_cur + pc));
    if (threadIdx.x == 0 && p.ss_done) *p.ss_done = done;
}

size_t coarse_strips_bytes(int nx, int ny, int nz) {
    return (size_t)3 * (size_t)(nx + 8) * (ny + 2) * (nz + 2) * sizeof(float);
}

template <typename T>
size_t coarse_small_bytes(int nx, int ny, int nz) {
    return (size_t)3 * (size_t)(nx + 2) * (ny + 2) * (nz + 2) * sizeof(T);
}

}  // namespace

template <typename T>
size_t coarse_smem_bytes(long long n) {
    return (size_t)(4 * n) * sizeof(T);
}

template <typename T>
bool coarse_fits(long long n) {
    // shared-memory capacity, the per-thread cell table, and 10-bit packed coordinates
    return coarse_smem_bytes<T>(n) <= kSmemLimit && n <= (long long)kMaxCells * kCoarseThreads;
}

template <typename T>
cudaError_t launch_coarse_solve(const CoarseParams& p, cudaStream_t st) {
    const long long n = (long long)p.g.nx * p.g.ny * p.g.nz;
    const size_t bytes = coarse_smem_bytes<T>(n);
    if (bytes > kSmemLimit) return cudaErrorInvalidValue;
    int threads = kCoarseThreads;
    if (n < threads) threads = (int)((n + 31) / 32) * 32;
    if constexpr (std::is_same<T, float>::value) {
        const size_t sb = coarse_strips_bytes(p.g.nx, p.g.ny, p.g.nz);
        const bool aligned = ((reinterpret_cast<uintptr_t>(p.rhs) | reinterpret_cast<uintptr_t>(p.u_out)) & 15) == 0;
        if ((p.g.nx & 3) == 0 && n / 4 <= kCoarseThreads && sb <= kSmemLimit && aligned) {
            const int strips = (int)(n / 4);
            k_coarse_strips<<<1, ((strips + 31) / 32) * 32, sb, st>>>(p);
            return cudaGetLastError();
        }
    }
    const size_t small = coarse_small_bytes<T>(p.g.nx, p.g.ny, p.g.nz);
    if (n <= kSmallCells && small <= kSmemLimit) {
        k_coarse_small<T><<<1, threads, small, st>>>(p);
        return cudaGetLastError();
    }
    if (n <= 4LL * kCoarseThreads) k_coarse_solve<T, 4><<<1, threads, bytes, st>>>(p);
    else k_coarse_solve<T, kMaxCells><<<1, threads, bytes, st>>>(p);
    return cudaGetLastError();
}

cudaError_t coarse_configure() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_coarse_strips, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmemLimit)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_coarse_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmemLimit)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_coarse_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmemLimit)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_coarse_solve<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmemLimit)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_coarse_solve<float, kMaxCells>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_coarse_solve<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmemLimit)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_coarse_solve<double, kMaxCells>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemLimit);
}

template size_t coarse_smem_bytes<float>(long long);
template size_t coarse_smem_bytes<double>(long long);
template bool coarse_fits<float>(long long);
template bool coarse_fits<double>(long long);
template cudaError_t launch_coarse_solve<float>(const CoarseParams&, cudaStream_t);
template cudaError_t launch_coarse_solve<double>(const CoarseParams&, cudaStream_t);

}  // namespace sg
