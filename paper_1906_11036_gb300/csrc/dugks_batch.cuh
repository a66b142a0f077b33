// dugks_batch.cuh -- many independent NCDE instances (uneven grid sizes and
// coefficients) advanced by one persistent launch per time step.
//
// Every instance is cut into tiles (30-column strip x row segment), the same
// unit the single-instance fused step gives one warp.  A launch holds as many
// one-warp CTAs as fit on the GPU; each warp takes tiles from a global
// counter (largest instances first) and runs the single-precision row
// routine of the single-instance step (sv_rows) on them, carrying its TMA
// stage ring from one tile to the next, so every instance's result is the
// single-instance step's bit for bit.  Instances step in lockstep, so one parity selects the
// source buffer of every instance.
#pragma once
#include "dugks_step_vp.cuh"

namespace dugks {

template <int NC>
struct BatchInst {
    CUtensorMap tmap[2];          // 3-D descriptors of the instance's two ftilde buffers
    StepArgs<float, NC> args[2];  // args[p] reads buffer p and writes buffer 1 - p
    ConstsP<NC> k;
    const RowY* rw;  // per-row y metrics of the instance
    int seg_rows, nstrips, nseg, tile_begin;
};

// resident warps per SM the batched kernel is compiled for (its register budget)
#ifndef DUGKS_BATCH_MIN_WARPS
#define DUGKS_BATCH_MIN_WARPS 12
#endif

template <int NC>
__global__ void __launch_bounds__(32, DUGKS_BATCH_MIN_WARPS)
    batch_step_vp(const BatchInst<NC>* __restrict__ insts, const int* __restrict__ tile_inst, const int ntiles,
                  const int parity, int* __restrict__ counter, const int S, int* __restrict__ err) {
    using L = WarpLayout<float>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(S) * L::STAGE_BYTES);
    const int lane = threadIdx.x;
    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncwarp();
    int ring = 0;
    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        if (*reinterpret_cast<volatile int*>(err) != 0) break;  // a bounded wait expired somewhere
        const BatchInst<NC>& I = insts[tile_inst[t]];
        const int local = t - I.tile_begin;
        const int strip = local % I.nstrips, seg = local / I.nstrips;
        const StepArgs<float, NC>& a = I.args[parity];
        const int xw = strip * L::WI;
        const int y0 = seg * I.seg_rows;
        const int y1 = min(y0 + I.seg_rows, a.ny);
        const bool edge = xw - 1 < 0 || xw + L::WI >= a.nx;
        const bool yg = !a.yper && (y0 == 0 || y1 == a.ny);
        sv_rows<NC>(&I.tmap[parity], a, I.k, I.rw, smem, bars, S, lane, xw, y0, y1, edge, yg, ring);
    }
}

}  // namespace dugks
