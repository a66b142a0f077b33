// dugks_batch.cuh -- many independent NCDE instances (uneven grid sizes and
// coefficients) advanced by one persistent launch per time step.
//
// Every instance is cut into tiles (30-column strip x row segment), the same
// unit the single-instance fused step gives one warp: long segments over most
// of its rows, short ones over the rest, the short tiles of every instance
// queued after all the long ones so that they even out the end of the launch.
// A launch holds as many one-warp CTAs as fit on the GPU; each warp takes
// tiles from a global counter (largest instances first) and runs the single-precision row
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
};

// one tile of the queue: instance, strip, rows y0 .. y1-1
struct BatchTile {
    int inst, strip, y0, y1;
};

// resident warps per SM the batched kernel is compiled for (its register budget)
// (the instance's arguments and constants are staged in shared memory per tile, so the row
// routine fits 16 warps per SM: 256 batched instances 0.498 ms per step against 0.559 ms
// with them held in registers at 12 warps per SM)
#ifndef DUGKS_BATCH_MIN_WARPS
#define DUGKS_BATCH_MIN_WARPS 16
#endif
#ifndef DUGKS_BATCH_SMEM_CONSTS
#define DUGKS_BATCH_SMEM_CONSTS 1
#endif

template <int NC>
__global__ void __launch_bounds__(32, DUGKS_BATCH_MIN_WARPS)
    batch_step_vp(const BatchInst<NC>* __restrict__ insts, const BatchTile* __restrict__ tiles, const int ntiles,
                  const int parity, int* __restrict__ counter, const int S, int* __restrict__ err) {
    using L = WarpLayout<float>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(S) * L::STAGE_BYTES);
#if DUGKS_BATCH_SMEM_CONSTS
    __shared__ __align__(16) StepArgs<float, NC> sargs[1];
    __shared__ __align__(16) ConstsP<NC> sk[1];
#endif
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
        const BatchTile tl = tiles[t];
        const BatchInst<NC>& I = insts[tl.inst];
#if DUGKS_BATCH_SMEM_CONSTS
        // the instance's step arguments and constants, staged in this warp's shared memory: the
        // row routine then re-reads them after each row's wait instead of holding them in registers
        {
            const uint32_t* src0 = reinterpret_cast<const uint32_t*>(&I.args[parity]);
            const uint32_t* src1 = reinterpret_cast<const uint32_t*>(&I.k);
            uint32_t* d0 = reinterpret_cast<uint32_t*>(sargs);
            uint32_t* d1 = reinterpret_cast<uint32_t*>(sk);
            __syncwarp();
            for (int q = lane; q < int(sizeof(StepArgs<float, NC>) / 4); q += 32) d0[q] = src0[q];
            for (int q = lane; q < int(sizeof(ConstsP<NC>) / 4); q += 32) d1[q] = src1[q];
            __syncwarp();
        }
        const StepArgs<float, NC>& a = *sargs;
        const ConstsP<NC>& kk = *sk;
#else
        const StepArgs<float, NC>& a = I.args[parity];
        const ConstsP<NC>& kk = I.k;
#endif
        const int xw = tl.strip * L::WI;
        const int y0 = tl.y0, y1 = tl.y1;
        const bool edge = xw - 1 < 0 || xw + L::WI >= a.nx;
        const bool yg = !a.yper && (y0 == 0 || y1 == a.ny);
        sv_rows<NC>(&I.tmap[parity], a, kk, I.rw, smem, bars, S, lane, xw, y0, y1, edge, yg, ring);
    }
}

}  // namespace dugks
