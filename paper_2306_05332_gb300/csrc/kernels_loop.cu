// The outer convergence loop of Sec. 2.1 on the device: V-cycles repeat while
// the relative residual ||L phi - f|| / ||L 0 - f|| is above the tolerance
// (Sec. 4.1), decided by one-thread kernels that set the conditions of the
// WHILE nodes of a CUDA graph, so a solve (or a batch of them) runs without a
// host round trip per cycle.  The decisions are those of the host loop:
//   * after each cycle: the relative residual (mixed precision: of the FP64
//     residual carried by recurrence), its history, the coarse super-steps;
//   * mixed precision, when the recurrence meets the tolerance: leave the
//     inner loop so that the true FP64 residual is computed once and
//     confirmed (or the cycles resume from it);
//   * a non-finite residual, the cycle cap or a fixed cycle count end it.
#include "sg_internal.cuh"

namespace sg {

namespace {

__device__ __forceinline__ bool loop_met(const DeviceLoop& d, double rel, double maxabs) {
    return d.mtol > 0.0 ? maxabs <= d.mtol : rel <= d.tol;
}

__device__ __forceinline__ double loop_rel(const DeviceLoop& d, const Reduced& r) {
    return sqrt(r.sumsq / d.nn) / d.rden;
}

__device__ __forceinline__ void loop_record(DeviceLoop& d, double rel, double maxabs) {
    if (d.m < kLoopHistory) d.history[d.m] = rel;
    d.rel = rel;
    d.maxabs = maxabs;
}

// After a cycle: count it and decide whether the inner loop runs another.
__global__ void k_loop_step(DeviceLoop* dl, const Reduced* red, const int* ss_done, const int* sched,
                            cudaGraphConditionalHandle inner) {
    DeviceLoop& d = *dl;
    const int ss = ss_done ? *ss_done : 0;
    if (d.m < kLoopHistory) d.coarse_ss[d.m] = ss;
    long long cs = 0;
    for (int q = 0; q < ss && q < d.sched_len; ++q) cs += sched[q];
    d.coarse_stage_cells += cs * d.coarse_cells;
    d.m += 1;
    const double rel = loop_rel(d, *red), maxabs = red->maxabs;
    const bool finite = isfinite(rel);
    unsigned go = 0;
    if (!d.fixed && finite && loop_met(d, rel, maxabs) && d.confirm) {
        d.pending = 1;                      // the true residual decides (loop_confirm)
    } else {
        loop_record(d, rel, maxabs);
        if (!finite) d.status = kLoopNonFinite;
        else if (!d.fixed && loop_met(d, rel, maxabs)) d.status = kLoopDone;
        else if (d.m >= d.limit) d.status = d.fixed ? kLoopDone : kLoopNotConverged;
        else go = 1;
    }
    cudaGraphSetConditional(inner, go);
}

// After the inner loop (mixed precision: the true FP64 residual is in red):
// confirm, or resume the cycles.
__global__ void k_loop_confirm(DeviceLoop* dl, const Reduced* red, cudaGraphConditionalHandle outer,
                               cudaGraphConditionalHandle inner) {
    DeviceLoop& d = *dl;
    unsigned go = 0;
    d.confirms += 1;
    if (d.pending) {
        d.pending = 0;
        const double rel = loop_rel(d, *red), maxabs = red->maxabs;
        loop_record(d, rel, maxabs);
        if (!isfinite(rel)) d.status = kLoopNonFinite;
        else if (loop_met(d, rel, maxabs)) d.status = kLoopDone;
        else if (d.m >= d.limit) d.status = kLoopNotConverged;
        else go = 1;
    }
    cudaGraphSetConditional(inner, go);
    cudaGraphSetConditional(outer, go);
}

// Before the loop: both conditions from the state the host wrote (a solve
// already finished at its first residual runs no cycle).
__global__ void k_loop_init(const DeviceLoop* dl, cudaGraphConditionalHandle outer, cudaGraphConditionalHandle inner) {
    const unsigned go = dl->status == kLoopRunning ? 1u : 0u;
    cudaGraphSetConditional(outer, go);
    cudaGraphSetConditional(inner, go);
}

}  // namespace

cudaError_t launch_loop_init(const DeviceLoop* d, cudaGraphConditionalHandle outer, cudaGraphConditionalHandle inner,
                             cudaStream_t st) {
    k_loop_init<<<1, 1, 0, st>>>(d, outer, inner);
    return cudaGetLastError();
}

cudaError_t launch_loop_step(DeviceLoop* d, const Reduced* red, const int* ss_done, const int* sched,
                             cudaGraphConditionalHandle inner, cudaStream_t st) {
    k_loop_step<<<1, 1, 0, st>>>(d, red, ss_done, sched, inner);
    return cudaGetLastError();
}

cudaError_t launch_loop_confirm(DeviceLoop* d, const Reduced* red, cudaGraphConditionalHandle outer,
                                cudaGraphConditionalHandle inner, cudaStream_t st) {
    k_loop_confirm<<<1, 1, 0, st>>>(d, red, outer, inner);
    return cudaGetLastError();
}

}  // namespace sg
