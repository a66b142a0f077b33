// dugks_adjoint_rows.cuh -- the adjoint of one FP32 DUGKS step (reverse mode
// of the step of Section 2, arXiv:1906.11036) as a row march, for grids that
// are periodic on both axes.
//
// The arithmetic is that of adj_tile_kernel (same face adjoints, same
// transposed weights), reorganised like the forward step: one warp owns a
// strip of 28 columns (lanes 2..29; lanes 0, 1, 30, 31 are halo columns, two
// on each side because a y-face adjoint needs the x-slope of its cell) and
// marches up a row segment.  Rows of ftilde^n and mu arrive by TMA into a
// private ring of stages.  Instead of gathering the adjoint of P from stored
// face adjoints, every face scatters its contributions as soon as it is
// formed: into three rolling accumulators Pb for the rows n-2, n-1, n (this
// lane's and, through a shuffle, the neighbour lane's).  When the new row n has
// been processed, row n-2 has received every contribution (x-faces of rows
// n-3..n-1, y-faces below and above it) and is finished (Eqs. 2.21, 2.13
// transposed), and its stage is refilled.
#pragma once
#include "dugks_adjoint.cuh"

namespace dugks {

#ifndef DUGKS_ADJ_ROWS_MIN_WARPS
#define DUGKS_ADJ_ROWS_MIN_WARPS 16  // 126 registers, no spills; 4 stages keep 16 warps in shared memory
#endif

struct AdjRowLayout {
    static constexpr int WI = 28;                       // owned columns per warp
    static constexpr int BOXW = 36;                     // 32 columns from (xw - 2) rounded down to 16 bytes
    static constexpr int BOX_BYTES = Q * BOXW * 4;      // one row of ftilde or mu
    static constexpr int MU_OFF = ((BOX_BYTES + 127) / 128) * 128;
    static constexpr int STAGE_BYTES = 2 * MU_OFF;      // ftilde row, then mu row
    static size_t bytes(int stages) { return size_t(stages) * (STAGE_BYTES + 8) + 128; }
};

// S: ring stages (a power of two keeps the stage index a mask); WU: also form the u-derivative
template <int NC, int S, bool WU>
__global__ void __launch_bounds__(32, DUGKS_ADJ_ROWS_MIN_WARPS)
    adj_rows_kernel(const __grid_constant__ CUtensorMap tf, const __grid_constant__ CUtensorMap tmu,
                    const StepArgs<float, NC> a, const Consts<float, NC> k, const AdjConsts<float, NC> ka,
                    const AdjArgs<float> g, const int seg_rows) {
    static_assert(S >= 3, "the ring holds rows n - 2 .. n");
    using L = AdjRowLayout;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* stages = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(stages + size_t(S) * L::STAGE_BYTES);
    const int lane = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const int xw = blockIdx.x * L::WI;
    const int y0 = blockIdx.y * seg_rows;
    if (y0 >= ny || xw >= nx) return;
    const int y1 = min(y0 + seg_rows, ny);
    const long long cplane = (long long)nx * ny;
    const int j = xw - 2 + lane;                // this lane's column (periodic image when outside)
    const int jw = ((j % nx) + nx) % nx;
    const int xs = (xw - 2) & ~3;               // 16-byte aligned x of the box
    const bool from_smem = j >= 0 && j < nx;    // else read the periodic image from global memory
    const bool owner = lane >= 2 && lane <= 29 && j < nx;
    const int R = y1 - y0 + 4;                  // rows y0-2 .. y1+1
    auto wrow = [&](int r) { return r < 0 ? r + ny : (r >= ny ? r - ny : r); };  // r in [-2, ny + 1], ny >= 4

    // column metrics of this lane's cell and of its east face
    const FaceM<float> fE = a.fx[jw + 2];
    const CellM<float> cxj = a.cx[jw + 1], cxe = a.cx[((jw + 1) % nx) + 1];

    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](int t) {  // row y0 - 2 + t into stage t % S
        const int st = t % S, row = wrow(y0 - 2 + t);
        mbar_arrive_expect_tx(&bars[st], uint32_t(2 * L::BOX_BYTES));
        tma_load_3d(stages + size_t(st) * L::STAGE_BYTES, &tf, &bars[st], xs, row, 0);
        tma_load_3d(stages + size_t(st) * L::STAGE_BYTES + L::MU_OFF, &tmu, &bars[st], xs, row, 0);
    };
    if (lane == 0)
        for (int t = 0; t < min(S, R); ++t) issue(t);
    // row r's ftilde (which = 0) or mu (1): stage of row r, or the periodic image in global memory
    auto row_vals = [&](int r, int which, float (&v)[Q]) {
        const int t = r - (y0 - 2);
        if (from_smem) {
            const float* st = reinterpret_cast<const float*>(stages + size_t(t % S) * L::STAGE_BYTES +
                                                             (which ? L::MU_OFF : 0)) + (j - xs);
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i] = st[i * L::BOXW];
        } else {
            const float* src = (which ? g.mu : g.f) + (long long)wrow(r) * nx + jw;
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i] = src[i * cplane];
        }
    };

    float Pm2[Q], Pm1[Q], Pn[Q];  // P = fbar^+ of rows n-2, n-1, n (this lane's column)
    float Ba[Q], Bb[Q], Bc[Q];    // adjoint of P accumulated for rows n-2, n-1, n
#pragma unroll
    for (int i = 0; i < Q; ++i) Pm2[i] = Pm1[i] = Pn[i] = Ba[i] = Bb[i] = Bc[i] = 0.f;
    double djdl = 0.0, du[2] = {0.0, 0.0};
    bool failed = false;
    int t = 0;
    for (; t < R; ++t) {
        const int n = y0 - 2 + t;
        const bool ok = mbar_wait_bounded(&bars[t % S], uint32_t((t / S) & 1), 2000000000ull);
        if (__any_sync(0xffffffffu, !ok)) { failed = true; break; }
        // P of the new row (Eq. 2.21; periodic, no ghosts)
        {
            float ft[Q], fe[Q];
            row_vals(n, 0, ft);
            float phi = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) phi += ft[i];
            feq_all(k, phi, fe);
#pragma unroll
            for (int i = 0; i < Q; ++i) Pn[i] = fmaf(k.a_bp, ft[i], k.b_bp * fe[i]);
        }
        float mq[Q];  // mu of row n - 1
        if (n >= y0) row_vals(n - 1, 1, mq);
        if (n >= y0) {
            // x-face east of this lane's cell in row q = n - 1 (faces of rows y0-1 .. y1)
            const int q = n - 1;
            const float igq = a.cy[wrow(q) + 1].ig;
            float Gy[Q], fb[Q], A[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) Gy[i] = EY(i) != 0 ? (Pn[i] - Pm2[i]) * igq : 0.f;
            float phib = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float en = float(EX(i)), et = float(EY(i));
                const float PR = __shfl_down_sync(0xffffffffu, Pm1[i], 1);
                const float GR = EY(i) != 0 ? __shfl_down_sync(0xffffffffu, Gy[i], 1) : 0.f;
                fb[i] = ((1.f - fE.w) + en * fE.hcd) * Pm1[i] - et * k.hc * fE.tl * Gy[i] +
                        (fE.w - en * fE.hcd) * PR - et * k.hc * fE.tr * GR;
                phib += fb[i];
            }
            float gv[Q], fe[Q];
            float sg = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                gv[i] = 0.f;
                fe[i] = 0.f;
                if (EX(i) != 0) {
                    const float muR = __shfl_down_sync(0xffffffffu, mq[i], 1);
                    gv[i] = float(EX(i)) * (cxe.r * muR - cxj.r * mq[i]);
                    fe[i] = feq_i(k, i, phib);
                    sg += gv[i] * dfeq_i(ka, i, phib);
                }
            }
            float sdl = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                A[i] = fmaf(ka.a_f, gv[i], ka.b_f * sg);
                if (EX(i) != 0) sdl += gv[i] * fmaf(ka.da_f, fb[i], ka.db_f * fe[i]);
            }
            if (owner && q >= y0 && q < y1) {
                djdl += double(sdl);
                if (WU) {  // Eq. 2.22: b_f feq(phi_b) of the crossing velocities
                    float w[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) w[i] = ka.b_f * gv[i];
                    add_du(ka, phib, w, xmask(), du);
                }
            }
            // scatter: normal weights into row q of this lane (L) and of the east lane (R);
            // tangential slope weights into rows q + 1 and q - 1 of both
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                Bb[i] = fmaf((1.f - fE.w) + float(EX(i)) * fE.hcd, A[i], Bb[i]);
                const float rs = __shfl_up_sync(0xffffffffu, (fE.w - float(EX(i)) * fE.hcd) * A[i], 1);
                Bb[i] += rs;
                if (EY(i) != 0) {
                    const float c = -float(EY(i)) * k.hc * igq * A[i];
                    const float tL = c * fE.tl;
                    const float tR = __shfl_up_sync(0xffffffffu, c * fE.tr, 1);
                    Bc[i] += tL + tR;
                    Ba[i] -= tL + tR;
                }
            }
        }
        if (n >= y0 && n <= y1) {
            // y-face between rows n - 1 and n of this lane's column (faces y0 .. y1)
            const FaceM<float> m = a.fy[n + 1];
            const float ig = cxj.ig;
            float mn[Q], fb[Q], A[Q];
            row_vals(n, 1, mn);
            float phib = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float en = float(EY(i)), et = float(EX(i));
                float GL = 0.f, GR = 0.f;  // x-slopes of the cells below and above the face
                if (EX(i) != 0) {
                    GL = (__shfl_down_sync(0xffffffffu, Pm1[i], 1) - __shfl_up_sync(0xffffffffu, Pm1[i], 1)) * ig;
                    GR = (__shfl_down_sync(0xffffffffu, Pn[i], 1) - __shfl_up_sync(0xffffffffu, Pn[i], 1)) * ig;
                }
                fb[i] = ((1.f - m.w) + en * m.hcd) * Pm1[i] - et * k.hc * m.tl * GL + (m.w - en * m.hcd) * Pn[i] -
                        et * k.hc * m.tr * GR;
                phib += fb[i];
            }
            const float rL = a.cy[wrow(n - 1) + 1].r, rR = a.cy[wrow(n) + 1].r;
            float gv[Q], fe[Q];
            float sg = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                gv[i] = 0.f;
                fe[i] = 0.f;
                if (EY(i) != 0) {
                    gv[i] = float(EY(i)) * (rR * mn[i] - rL * mq[i]);
                    fe[i] = feq_i(k, i, phib);
                    sg += gv[i] * dfeq_i(ka, i, phib);
                }
            }
            float sdl = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                A[i] = fmaf(ka.a_f, gv[i], ka.b_f * sg);
                if (EY(i) != 0) sdl += gv[i] * fmaf(ka.da_f, fb[i], ka.db_f * fe[i]);
            }
            if (owner && n < y1) {
                djdl += double(sdl);
                if (WU) {
                    float w[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) w[i] = ka.b_f * gv[i];
                    add_du(ka, phib, w, ymask(), du);
                }
            }
            // scatter: normal weights into rows n - 1 (L) and n (R) of this lane; x-slope weights
            // into the same rows of the lanes to the east (+) and west (-)
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                Bb[i] = fmaf((1.f - m.w) + float(EY(i)) * m.hcd, A[i], Bb[i]);
                Bc[i] = fmaf(m.w - float(EY(i)) * m.hcd, A[i], Bc[i]);
                if (EX(i) != 0) {
                    const float c = -float(EX(i)) * k.hc * ig * A[i];
                    const float uL = c * m.tl, uR = c * m.tr;
                    Bb[i] += __shfl_up_sync(0xffffffffu, uL, 1) - __shfl_down_sync(0xffffffffu, uL, 1);
                    Bc[i] += __shfl_up_sync(0xffffffffu, uR, 1) - __shfl_down_sync(0xffffffffu, uR, 1);
                }
            }
        }
        if (n >= y0 + 2) {
            // row n - 2 has every contribution: transpose Eqs. 2.21 and 2.13 and phi = sum f
            const int r = n - 2;
            float ft[Q], mu[Q], fe[Q], dfe[Q];
            row_vals(r, 0, ft);
            row_vals(r, 1, mu);
            float phi = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) phi += ft[i];
            feq_all(k, phi, fe);
            dfeq_all(ka, phi, dfe);
            float phibar = 0.f, s = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                phibar += (ka.b_bp * Ba[i] + ka.b_tp * mu[i]) * dfe[i];
                s += Ba[i] * fmaf(ka.da_bp, ft[i], ka.db_bp * fe[i]) + mu[i] * fmaf(ka.da_tp, ft[i], ka.db_tp * fe[i]);
            }
            if (owner) {
                djdl += double(s);
                if (WU) {  // Eqs. 2.21 and 2.13: b_bp feq(phi) in P and b_tp feq(phi) in ftilde^+
                    float w[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) w[i] = fmaf(ka.b_bp, Ba[i], ka.b_tp * mu[i]);
                    add_du(ka, phi, w, kAllQ, du);
                }
                float* out = g.lam + (long long)r * nx + j;
#pragma unroll
                for (int i = 0; i < Q; ++i) out[i * cplane] = fmaf(ka.a_bp, Ba[i], fmaf(ka.a_tp, mu[i], phibar));
            }
        }
        // the stage of row n - 2 is no longer read: refill it
        __syncwarp();
        if (n >= y0 && lane == 0 && t - 2 + S < R) {
            fence_proxy_async_smem();
            issue(t - 2 + S);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            Pm2[i] = Pm1[i];
            Pm1[i] = Pn[i];
            Ba[i] = Bb[i];
            Bb[i] = Bc[i];
            Bc[i] = 0.f;
        }
    }
    if (failed && lane == 0) {
        atomicOr(a.err, 1);
        // let the copies still in flight land before the warp exits: rows t .. issued - 1
        const int released = max(0, t - 2);
        const int issued = min(R, released + S);
        for (int u = t; u < issued; ++u) mbar_wait_bounded(&bars[u % S], uint32_t((u / S) & 1), 100000000ull);
    }
    __syncwarp();
    const double v[3] = {djdl, du[0], du[1]};
    block_partial3(v, g.partial + blockIdx.y * gridDim.x + blockIdx.x, g.pstride, g.accumulate);
}

}  // namespace dugks
