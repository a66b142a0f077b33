// dugks_step_vp.cuh -- the production single-precision DUGKS step for D2Q9
// (arXiv:1906.11036, Section 2, the step summary at the end of the section).
//
// One warp owns a strip of 30 interior columns (lane l holds column
// xw - 1 + l; lanes 0 and 31 are the halo columns) and a segment of rows, and
// marches up the segment one row at a time.  Each row of ftilde (nine
// planes, 36 columns) arrives in shared memory by one 3-D TMA copy into a
// ring of S stages guarded by bounded mbarrier waits; ftilde is read once
// from HBM and the new state written once.  Per row r the warp
//
//   1. forms P = fbar^+ (Eq. 2.21), ftilde^+ (Eq. 2.13 in the form of
//      Eq. 2.23) and the moments of P: phi = sum_i P_i (= sum_i ftilde_i),
//      Mx = sum_i e_x,i P_i, My = sum_i e_y,i P_i;
//   2. takes x-slopes of P by warp shuffles and completes the y-face below
//      row r (Eqs. 2.19, 2.20, 2.26): fbar of the velocities that cross it,
//      and phi_b (text after Eq. 2.20) from the moments of its two cells;
//   3. forms the original distribution at that face (Eq. 2.22) and its flux;
//   4. completes the x-faces of row r - 1 the same way (y-slopes from rows
//      r - 2 and r) and writes the update of row r - 1 (Eq. 2.12).
//
// phi_b from moments: the face value fbar_i is linear in P of the two cells
// and in their tangential slopes, so its sum over i is the same linear form
// in (phi, Mx, My) and in the slope of the tangential moment; velocities that
// do not cross a face enter only through that sum, so their fbar is never
// formed.  The update of a row is carried as U = ftilde^+ plus the flux of
// the face below it, so the south-face flux is not kept separately.
//
// The nine velocities are packed as the opposite pairs q = (1,3), (2,4),
// (5,7), (6,8) plus the rest velocity on the packed FP32 instructions of
// sm_100+ (__ffma2_rn, __fadd2_rn, __fmul2_rn).
#pragma once
#include "dugks_kernels.cuh"

namespace dugks {

// Metrics of row k of a rectilinear mesh, precomputed on the host (Eqs. 2.19,
// 2.20 with the reconstruction weights of the interface between two rows).
// Entry k + 1 of the array holds row k = -1 .. ny.
struct __align__(16) RowY {
    float2 up;  // the face below row k, seen from row k (its upper cell): (w - hcd, w + hcd)
    float u0;   // w  (velocities that do not move in y)
    float gu;   // h c tr: weight of row k's tangential slope at that face
    float2 lp;  // the face above row k, seen from row k (its lower cell): (1 - w + hcd, 1 - w - hcd)
    float l0;   // 1 - w
    float gl;   // h c tl
    float igy;  // 1 / (y_{k+1} - y_{k-1}): central-difference factor of row k
    float ry;   // dt c / dy_k: flux factor of the update of row k
    float hup;  // hcd of the face below row k
    float hlo;  // hcd of the face above row k
};

struct SvCell {
    V9 P;               // fbar^+ of the cell
    float phi, mx, my;  // sum_i P_i, sum_i e_x,i P_i, sum_i e_y,i P_i
};

__device__ __forceinline__ void sv_moments(SvCell& c) {
    const float d0 = c.P.p[0].v.x - c.P.p[0].v.y, d1 = c.P.p[1].v.x - c.P.p[1].v.y;
    const float d2 = c.P.p[2].v.x - c.P.p[2].v.y, d3 = c.P.p[3].v.x - c.P.p[3].v.y;
    c.mx = (d0 + d2) - d3;  // e_x of the pairs' first velocities: +1, 0, +1, -1
    c.my = (d1 + d2) + d3;  // e_y: 0, +1, +1, +1
}

// P (Eq. 2.21 with b_bp folded into the equilibrium polynomials), Fp = P + (P - ftilde)/3
// (Eq. 2.23) and the moments.  sum_i P_i = phi: the weights of Eq. 2.21 sum to one and the
// rest velocity takes the zeroth moment of Eq. 2.7.
template <int NC>
__device__ __forceinline__ void sv_cell(const ConstsP<NC>& k, const V9& F, SvCell& c, V9& Fp) {
    const float phi = vsum(F);
    const F2 phi2 = f2(phi);
    F2 hs = f2(0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const F2 h = hbp2(k, q, phi2);
        c.P.p[q] = fma2(F2{k.a_bp2}, F.p[q], h);
        hs = hs + h;
    }
    c.P.z = fmaf(k.a_bp, F.z, fmaf(k.b_bp, phi, -(hs.v.x + hs.v.y)));
#pragma unroll
    for (int q = 0; q < 4; ++q) Fp.p[q] = fma2(F2{k.third2}, c.P.p[q] - F.p[q], c.P.p[q]);
    Fp.z = fmaf(k.third, c.P.z - F.z, c.P.z);
    c.phi = phi;
    sv_moments(c);
}

// Mirrored ghost at a Dirichlet wall with value bv (non-equilibrium extrapolation):
// phi_g = 2 bv - phi, P_g = feq(phi_g) + (P - feq(phi)); its moments follow.
template <int NC>
__device__ __forceinline__ void sv_ghost(const ConstsP<NC>& k, SvCell& c, const float bv) {
    const float phig = 2.f * bv - c.phi;
    const F2 x = f2(c.phi), xg = f2(phig);
    F2 s = f2(0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        F2 a = f2(k.s.feq[PA(q)][NC - 1], k.s.feq[PB(q)][NC - 1]), b = a;
#pragma unroll
        for (int m = NC - 2; m >= 0; --m) {
            const F2 cm = f2(k.s.feq[PA(q)][m], k.s.feq[PB(q)][m]);
            a = fma2(a, xg, cm);
            b = fma2(b, x, cm);
        }
        const F2 d = a - b;
        c.P.p[q] = c.P.p[q] + d;
        s = s + d;
    }
    c.P.z += (phig - c.phi) - (s.v.x + s.v.y);  // rest velocity: zeroth moment
    c.phi = phig;
    sv_moments(c);
}

// Rows y0-1 .. y1 of one strip pass through this warp's ring; rows y0 .. y1-1 are
// updated.  EDGE: the strip touches the first or last column (ghost, periodic-image or
// idle lanes).  YG: the segment may meet a Dirichlet wall in y (ghost rows -1 and ny).
// Both are warp-uniform run-time flags: a loop over segments then holds one copy of
// the routine (several inlined copies in one loop exhaust the register budget).  PLAIN: a
// warp that meets neither (known at compile time), so the flags and their branches fold away.
// `ring` counts the rows this warp already passed through its ring (row t of the warp
// uses stage t % S in phase (t / S) & 1), so a warp may run several segments.
template <int NC, bool PLAIN = false>
__device__ __forceinline__ void sv_rows(const CUtensorMap* tin, const StepArgs<float, NC>& a, const ConstsP<NC>& k,
                                        const RowY* __restrict__ rw, unsigned char* stages, uint64_t* bars,
                                        const int S, const int lane, const int xw, const int y0, const int y1,
                                        const bool edge_in, const bool yg_in, int& ring) {
    using L = WarpLayout<float>;
    const bool EDGE = PLAIN ? false : edge_in, YG = PLAIN ? false : yg_in;
    const int nx = a.nx, ny = a.ny;
    const int j = xw - 1 + lane;
    const int xs = (xw - 1) & ~(L::ALIGN - 1);
    const int R = y1 - y0 + 2;

    int role = ROLE_IN, scol = j;
    if (EDGE) {
        if (j >= 0 && j < nx) { role = ROLE_IN; scol = j; }
        else if (j == -1) { role = a.xper ? ROLE_WRAP_W : ROLE_GHOST_W; scol = a.xper ? nx - 1 : 0; }
        else if (j == nx) { role = a.xper ? ROLE_WRAP_E : ROLE_GHOST_E; scol = a.xper ? 0 : nx - 1; }
        else { role = ROLE_OUT; scol = 0; }
    }
    const bool from_smem = !EDGE || role == ROLE_IN || role == ROLE_GHOST_W || role == ROLE_GHOST_E;
    const bool ghost_col = EDGE && (role == ROLE_GHOST_W || role == ROLE_GHOST_E);
    const bool no_slope = EDGE && (ghost_col || role == ROLE_OUT);  // y-slopes weighted by zero: kept finite
    const bool updates = (!EDGE || role == ROLE_IN) && lane >= 1 && lane <= L::WI;
    const int jm = EDGE ? min(max(j, -1), nx) : j;
    const FaceM<float> fW = a.fx[jm + 1], fE = a.fx[jm + 2];
    const CellM<float> cxj = a.cx[jm + 1];
    const float bvx = role == ROLE_GHOST_W ? k.s.bcv[0] : k.s.bcv[1];
    const int soff = scol - xs;

    // x-face weights of this cell for the pairs that cross x-faces: q0, q2 (first velocity +x), q3 (-x)
    const F2 axLp = sgn2(1.f - fE.w, fE.hcd, 1), axLn = sgn2(1.f - fE.w, fE.hcd, -1);
    const F2 axRp = sgn2(fW.w, -fW.hcd, 1), axRn = sgn2(fW.w, -fW.hcd, -1);
    const F2 gxL = sgn2(0.f, -k.hc * fE.tl, 1), gxR = sgn2(0.f, -k.hc * fW.tr, 1);
    const F2 rxp = sgn2(0.f, -cxj.r, 1), rxn = sgn2(0.f, -cxj.r, -1);
    // phi_b halves: this cell as the left cell of its east face, and as the right cell of its west face
    const float eL0 = 1.f - fE.w, eLx = fE.hcd, eLy = -k.hc * fE.tl;
    const float wR0 = fW.w, wRx = -fW.hcd, wRy = -k.hc * fW.tr;
    const float igx = cxj.ig;
    const float ymask = no_slope ? 0.f : 1.f;

    auto src_row = [&](int r) -> int {
        if (r < 0) return a.yper ? r + ny : 0;
        if (r >= ny) return a.yper ? r - ny : ny - 1;
        return r;
    };
    if (lane == 0) {
        for (int q = 0; q < min(S, R); ++q) {
            const int st = (ring + q) % S;
            mbar_arrive_expect_tx(&bars[st], uint32_t(L::BOX_BYTES));
            tma_load_3d(stages + size_t(st) * L::STAGE_BYTES, tin, &bars[st], xs, src_row(y0 - 1 + q), 0);
        }
    }
    int s = ring % S, issued = min(S, R), consumed = 0;
    uint32_t ph = uint32_t((ring / S) & 1);

    // next row of ftilde from the ring; refills the stage it frees
    auto load_row = [&](int r, V9& F) -> bool {
        const bool ok = mbar_wait_bounded(&bars[s], ph, 2000000000ull);
        if (__any_sync(0xffffffffu, !ok)) return false;
        float ft[Q];
        if (from_smem) {
            const float* st = reinterpret_cast<const float*>(stages + size_t(s) * L::STAGE_BYTES) + soff;
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = st[i * L::BOXW];
        } else if (role != ROLE_OUT) {
            const long long base = (long long)src_row(r) * a.pitch + scol;
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = a.fin[i * a.plane + base];
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) F.p[q] = f2(ft[PA(q)], ft[PB(q)]);
        F.z = ft[0];
        __syncwarp();
        if (issued < R) {
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[s], uint32_t(L::BOX_BYTES));
                tma_load_3d(stages + size_t(s) * L::STAGE_BYTES, tin, &bars[s], xs, src_row(r + S), 0);
            }
            ++issued;
        }
        if (++s == S) { s = 0; ph ^= 1u; }
        ++consumed;
        return true;
    };
    // row r's cell: P, Fp, moments; ghost columns and rows by the mirrored NEE ghost
    auto cell_row = [&](int r, const V9& F, SvCell& c, V9& Fp) {
        sv_cell(k, F, c, Fp);
        if (EDGE || YG) {
            const bool grow = YG && (r < 0 || r >= ny);
            if (ghost_col || grow) sv_ghost(k, c, ghost_col ? bvx : (r < 0 ? k.s.bcv[2] : k.s.bcv[3]));
        }
    };
    // x-slopes of q2 and q3 (the sign of q3, whose first velocity moves in -x, folded in) and of Mx;
    // zero on ghost rows, where the face weights give them no weight
    auto grad_x = [&](int r, const SvCell& c, F2& g2, F2& g3, float& gm) {
        const float ig = (YG && (r < 0 || r >= ny)) ? 0.f : igx;
        const F2 ig2 = f2(ig);
        g2 = (shfl_dn2(c.P.p[2]) - shfl_up2(c.P.p[2])) * ig2;
        g3 = (shfl_up2(c.P.p[3]) - shfl_dn2(c.P.p[3])) * ig2;
        gm = (__shfl_down_sync(0xffffffffu, c.mx, 1) - __shfl_up_sync(0xffffffffu, c.mx, 1)) * ig;
    };
    struct Low {  // lower half of a y-face: fbar parts of q1, q2, q3 and of phi_b
        F2 q1, q2, q3;
        float ph;
    };
    auto lower = [&](const RowY& w, const SvCell& c, const F2 g2, const F2 g3, const float gm, Low& lo) {
        const F2 gl = f2(-w.gl, w.gl);
        lo.q1 = F2{w.lp} * c.P.p[1];
        lo.q2 = fma2(gl, g2, F2{w.lp} * c.P.p[2]);
        lo.q3 = fma2(gl, g3, F2{w.lp} * c.P.p[3]);
        lo.ph = fmaf(w.l0, c.phi, fmaf(w.hlo, c.my, -w.gl * gm));
    };
    // the y-face below row r: original f (Eq. 2.22) of the pairs that cross it
    auto yface = [&](const RowY& w, const SvCell& c, const F2 g2, const F2 g3, const float gm, const Low& lo,
                     F2& f1, F2& f2q, F2& f3) {
        const F2 gu = f2(-w.gu, w.gu);
        const F2 b1 = fma2(F2{w.up}, c.P.p[1], lo.q1);
        const F2 b2 = fma2(gu, g2, fma2(F2{w.up}, c.P.p[2], lo.q2));
        const F2 b3 = fma2(gu, g3, fma2(F2{w.up}, c.P.p[3], lo.q3));
        const F2 pb = f2(lo.ph + fmaf(w.u0, c.phi, fmaf(-w.hup, c.my, -w.gu * gm)));
        f1 = fma2(F2{k.a_f2}, b1, hf2(k, 1, pb));
        f2q = fma2(F2{k.a_f2}, b2, hf2(k, 2, pb));
        f3 = fma2(F2{k.a_f2}, b3, hf2(k, 3, pb));
    };

    bool failed = false;
    // carried between rows: c0 = row r-1; pm2, pm3, mym = q2, q3 and My of row r-2;
    // U0 = ftilde^+ of row r-1 plus the flux of the face below it; lo = lower half of the
    // face above row r-1; ig0, ry0 = metrics of row r-1
    SvCell c0;
    V9 U0, F, Fp;
    Low lo;
    F2 pm2 = f2(0.f), pm3 = f2(0.f);
    float mym = 0.f, ig0 = 0.f, ry0 = 0.f;
    {
        const RowY w = rw[y0];  // row y0 - 1
        if (!load_row(y0 - 1, F)) failed = true;
        if (!failed) {
            F2 g2, g3;
            float gm;
            cell_row(y0 - 1, F, c0, Fp);
            grad_x(y0 - 1, c0, g2, g3, gm);
            lower(w, c0, g2, g3, gm, lo);
            pm2 = c0.P.p[2];
            pm3 = c0.P.p[3];
            mym = c0.my;
        }
    }
    if (!failed) {
        const RowY w = rw[y0 + 1];  // row y0
        if (!load_row(y0, F)) failed = true;
        if (!failed) {
            F2 g2, g3, f1, fq2, f3;
            float gm;
            cell_row(y0, F, c0, U0);
            grad_x(y0, c0, g2, g3, gm);
            yface(w, c0, g2, g3, gm, lo, f1, fq2, f3);
            const F2 ryp = sgn2(0.f, w.ry, 1);
            U0.p[1] = fma2(ryp, f1, U0.p[1]);
            U0.p[2] = fma2(ryp, fq2, U0.p[2]);
            U0.p[3] = fma2(ryp, f3, U0.p[3]);
            lower(w, c0, g2, g3, gm, lo);
            ig0 = w.igy;
            ry0 = w.ry;
        }
    }
    // steady state: row r enters, row r - 1 is updated
#pragma unroll 2
    for (int r = y0 + 1; r <= y1; ++r) {
        if (failed) break;
        const RowY w = rw[r + 1];  // issued before the wait: its latency hides behind it
        if (!load_row(r, F)) { failed = true; break; }
        SvCell c;
        F2 g2, g3, f1, fq2, f3;
        float gm;
        cell_row(r, F, c, Fp);
        grad_x(r, c, g2, g3, gm);
        yface(w, c, g2, g3, gm, lo, f1, fq2, f3);
        lower(w, c, g2, g3, gm, lo);
        // the x-face east of (j, r-1): pairs q0, q2, q3 (Eqs. 2.19, 2.20, 2.26, 2.22)
        const float igy = EDGE ? ig0 * ymask : ig0;
        const F2 igy2 = f2(igy);
        const F2 gy2 = (c.P.p[2] - pm2) * igy2, gy3 = (c.P.p[3] - pm3) * igy2;
        const float gmy = (c.my - mym) * igy;
        const F2 l0 = axLp * c0.P.p[0], r0 = axRp * c0.P.p[0];
        const F2 l2 = fma2(gxL, gy2, axLp * c0.P.p[2]), r2 = fma2(gxR, gy2, axRp * c0.P.p[2]);
        const F2 l3 = fma2(gxL, gy3, axLn * c0.P.p[3]), r3 = fma2(gxR, gy3, axRn * c0.P.p[3]);
        const float pl = fmaf(eL0, c0.phi, fmaf(eLx, c0.mx, eLy * gmy));
        const float pr = fmaf(wR0, c0.phi, fmaf(wRx, c0.mx, wRy * gmy));
        const F2 b0 = l0 + shfl_dn2(r0), b2 = l2 + shfl_dn2(r2), b3 = l3 + shfl_dn2(r3);
        const F2 pb = f2(pl + __shfl_down_sync(0xffffffffu, pr, 1));
        const F2 e0 = fma2(F2{k.a_f2}, b0, hf2(k, 0, pb));
        const F2 e2 = fma2(F2{k.a_f2}, b2, hf2(k, 2, pb));
        const F2 e3 = fma2(F2{k.a_f2}, b3, hf2(k, 3, pb));
        // east minus west flux (the west face is lane - 1's east face)
        const F2 d0 = e0 - shfl_up2(e0), d2 = e2 - shfl_up2(e2), d3 = e3 - shfl_up2(e3);
        // update of row r - 1 (Eq. 2.12): U0 - (dt c / dy) e_y f(face above) - (dt c / dx) e_x (fE - fW)
        const F2 ryn = sgn2(0.f, -ry0, 1);
        V9 o;
        o.z = U0.z;
        o.p[0] = fma2(rxp, d0, U0.p[0]);
        o.p[1] = fma2(ryn, f1, U0.p[1]);
        o.p[2] = fma2(rxp, d2, fma2(ryn, fq2, U0.p[2]));
        o.p[3] = fma2(rxn, d3, fma2(ryn, f3, U0.p[3]));
        if (updates) {
            float* out = a.fout + (long long)(r - 1) * a.pitch + j;
            out[0] = o.z;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                out[PA(q) * a.plane] = o.p[q].v.x;
                out[PB(q) * a.plane] = o.p[q].v.y;
            }
        }
        // row r: ftilde^+ plus the flux of the face below it
        const F2 ryp = sgn2(0.f, w.ry, 1);
        U0 = Fp;
        U0.p[1] = fma2(ryp, f1, U0.p[1]);
        U0.p[2] = fma2(ryp, fq2, U0.p[2]);
        U0.p[3] = fma2(ryp, f3, U0.p[3]);
        pm2 = c0.P.p[2];
        pm3 = c0.P.p[3];
        mym = c0.my;
        c0 = c;
        ig0 = w.igy;
        ry0 = w.ry;
    }
    if (failed && lane == 0) {
        // record the timeout; wait (bounded) for this warp's copies still in flight
        atomicOr(a.err, 1);
        for (int q = consumed; q < issued; ++q) {
            mbar_wait_bounded(&bars[s], ph, 100000000ull);
            if (++s == S) { s = 0; ph ^= 1u; }
        }
    }
    ring += issued;
    __syncwarp();
}

// resident warps per SM the step kernel is compiled for (its register budget)
#ifndef DUGKS_SV_MIN_WARPS
#define DUGKS_SV_MIN_WARPS 16
#endif

// Row segments of a strip: the first nlong are seg_long rows long, the rest seg_short
// (the last one clipped at ny).  Blocks run in launch order, so the long segments fill
// the GPU first and the short ones fill in as warps finish.
struct SegPlan {
    int seg_long, nlong, seg_short;
};
__device__ __forceinline__ void seg_rows_of(const SegPlan& sp, const int k, const int ny, int& y0, int& y1) {
    if (k < sp.nlong) {
        y0 = k * sp.seg_long;
        y1 = y0 + sp.seg_long;
    } else {
        y0 = sp.nlong * sp.seg_long + (k - sp.nlong) * sp.seg_short;
        y1 = y0 + sp.seg_short;
    }
    y1 = min(y1, ny);
}

// One one-warp CTA per (strip, row segment): blockIdx.x = strip, blockIdx.y = segment.
// IP: interior CTAs run the interior variant of the row routine.  The host takes it for plans
// with long segments (2048^2 tanh mesh: 65.8 -> 63.75 us); without it for grids of short uniform
// segments, where the second copy of the routine in the kernel costs more than it saves
// (1024^2 periodic, 16-row segments: 25.05 us without, 25.71 us with).
template <int NC, bool IP>
__global__ void __launch_bounds__(32, DUGKS_SV_MIN_WARPS)
    step_vp(const __grid_constant__ CUtensorMap tin, const StepArgs<float, NC> a, const ConstsP<NC> k,
            const RowY* __restrict__ rw, const SegPlan sp, const int S) {
    using L = WarpLayout<float>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned; the layout reserves 128 bytes of slack
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(S) * L::STAGE_BYTES);
    const int lane = threadIdx.x;
    const int xw = blockIdx.x * L::WI;
    int y0, y1;
    seg_rows_of(sp, int(blockIdx.y), a.ny, y0, y1);
    if (y0 >= a.ny || xw >= a.nx) return;
    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool edge = xw - 1 < 0 || xw + L::WI >= a.nx;
    const bool yg = !a.yper && (y0 == 0 || y1 == a.ny);
    int ring = 0;
    if (IP && !edge && !yg)
        sv_rows<NC, true>(&tin, a, k, rw, smem, bars, S, lane, xw, y0, y1, false, false, ring);
    else
        sv_rows<NC>(&tin, a, k, rw, smem, bars, S, lane, xw, y0, y1, edge, yg, ring);
}


// ---------------------------------------------------------------------------
// the same row routine with the source terms F and R
// ---------------------------------------------------------------------------
//
// The source distributions enter linearly (Eqs. 2.12 and 2.18; the reconstruction of
// Eqs. 2.19, 2.20 is the same for fbar^+, R and F), so they are added to P = fbar^+ and to
// ftilde^+ of each cell after Eq. 2.21 (add_source_vp); phi_b then takes the zeroth moment of
// P with its sources, and a ghost mirrors the cell's own phi and carries its sources.  The
// fields S_k and phi^{n-1} of a row arrive in a second TMA box in the same ring stage.  One
// loop over the rows y0-1 .. y1 whose first two passes skip what needs the rows below keeps
// one inlined copy of the source arithmetic (instruction-cache footprint).
template <int NC, bool PLAIN = false>
__device__ __forceinline__ void sv_rows_src(const CUtensorMap* tin, const CUtensorMap* taux,
                                            const StepArgs<float, NC>& a, const ConstsP<NC>& k,
                                            const RowY* __restrict__ rw, const SrcArgs<float>& sa,
                                            unsigned char* stages, uint64_t* bars, const int S, const int lane,
                                            const int xw, const int y0, const int y1, const bool edge_in,
                                            const bool yg_in) {
    const bool EDGE = PLAIN ? false : edge_in, YG = PLAIN ? false : yg_in;
    using L = WarpLayout<float>;
    const int nx = a.nx, ny = a.ny;
    const int j = xw - 1 + lane;
    const int xs = (xw - 1) & ~(L::ALIGN - 1);
    const int R = y1 - y0 + 2;

    int role = ROLE_IN, scol = j;
    if (EDGE) {
        if (j >= 0 && j < nx) { role = ROLE_IN; scol = j; }
        else if (j == -1) { role = a.xper ? ROLE_WRAP_W : ROLE_GHOST_W; scol = a.xper ? nx - 1 : 0; }
        else if (j == nx) { role = a.xper ? ROLE_WRAP_E : ROLE_GHOST_E; scol = a.xper ? 0 : nx - 1; }
        else { role = ROLE_OUT; scol = 0; }
    }
    const bool from_smem = !EDGE || role == ROLE_IN || role == ROLE_GHOST_W || role == ROLE_GHOST_E;
    const bool ghost_col = EDGE && (role == ROLE_GHOST_W || role == ROLE_GHOST_E);
    const bool no_slope = EDGE && (ghost_col || role == ROLE_OUT);
    const bool updates = (!EDGE || role == ROLE_IN) && lane >= 1 && lane <= L::WI;
    const bool has_src = !(EDGE && role == ROLE_OUT);
    const int jm = EDGE ? min(max(j, -1), nx) : j;
    const FaceM<float> fW = a.fx[jm + 1], fE = a.fx[jm + 2];
    const CellM<float> cxj = a.cx[jm + 1];
    const float bvx = role == ROLE_GHOST_W ? k.s.bcv[0] : k.s.bcv[1];
    const int soff = scol - xs;

    const F2 axLp = sgn2(1.f - fE.w, fE.hcd, 1), axLn = sgn2(1.f - fE.w, fE.hcd, -1);
    const F2 axRp = sgn2(fW.w, -fW.hcd, 1), axRn = sgn2(fW.w, -fW.hcd, -1);
    const F2 gxL = sgn2(0.f, -k.hc * fE.tl, 1), gxR = sgn2(0.f, -k.hc * fW.tr, 1);
    const F2 rxp = sgn2(0.f, -cxj.r, 1), rxn = sgn2(0.f, -cxj.r, -1);
    const float eL0 = 1.f - fE.w, eLx = fE.hcd, eLy = -k.hc * fE.tl;
    const float wR0 = fW.w, wRx = -fW.hcd, wRy = -k.hc * fW.tr;
    const float igx = cxj.ig;
    const float ymask = no_slope ? 0.f : 1.f;

    auto src_row = [&](int r) -> int {
        if (r < 0) return a.yper ? r + ny : 0;
        if (r >= ny) return a.yper ? r - ny : ny - 1;
        return r;
    };
    const int stride = sa.stage_bytes;  // ftilde box, then the box of the fields and phi^{n-1}
    const uint32_t txb = uint32_t(L::BOX_BYTES + sa.aux_box);
    auto issue = [&](int st, int row) {
        mbar_arrive_expect_tx(&bars[st], txb);
        tma_load_3d(stages + size_t(st) * stride, tin, &bars[st], xs, row, 0);
        tma_load_3d(stages + size_t(st) * stride + L::STAGE_BYTES, taux, &bars[st], xs, row, 0);
    };
    if (lane == 0)
        for (int q = 0; q < min(S, R); ++q) issue(q, src_row(y0 - 1 + q));
    int s = 0, issued = min(S, R), consumed = 0;
    uint32_t ph = 0u;
    float Av[9];  // this lane's S_k (0..nterms-1) and phi^{n-1} (8) of the row just loaded
#pragma unroll
    for (int q = 0; q < 9; ++q) Av[q] = 0.f;

    auto load_row = [&](int r, V9& F) -> bool {
        const bool ok = mbar_wait_bounded(&bars[s], ph, 2000000000ull);
        if (__any_sync(0xffffffffu, !ok)) return false;
        float ft[Q];
        if (from_smem) {
            const float* st = reinterpret_cast<const float*>(stages + size_t(s) * stride) + soff;
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = st[i * L::BOXW];
            // (a term beyond nterms reads the last field: its weights are zero)
            const float* ax = reinterpret_cast<const float*>(stages + size_t(s) * stride + L::STAGE_BYTES) + soff;
#pragma unroll
            for (int q = 0; q < 8; ++q) Av[q] = ax[min(q, sa.nterms - 1) * L::BOXW];
            Av[8] = ax[sa.nterms * L::BOXW];
        } else if (role != ROLE_OUT) {
            const long long base = (long long)src_row(r) * a.pitch + scol;
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = a.fin[i * a.plane + base];
#pragma unroll
            for (int q = 0; q < 8; ++q) Av[q] = sa.aux_in[min(q, sa.nterms - 1) * sa.aux_plane + base];
            Av[8] = sa.aux_in[sa.nterms * sa.aux_plane + base];
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) ft[i] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) F.p[q] = f2(ft[PA(q)], ft[PB(q)]);
        F.z = ft[0];
        __syncwarp();
        if (issued < R) {
            if (lane == 0) {
                fence_proxy_async_smem();
                issue(s, src_row(r + S));
            }
            ++issued;
        }
        if (++s == S) { s = 0; ph ^= 1u; }
        ++consumed;
        return true;
    };

    // row r's cell: P and Fp with the source terms, the mirrored ghost, the moments of P
    auto cell_row = [&](int r, const V9& F, SvCell& c, V9& Fp) {
        sv_cell(k, F, c, Fp);  // c.phi = sum_i ftilde_i of the cell
        if (has_src) {
            if (updates && r >= y0 && r < y1) sa.aux_out[sa.nterms * sa.aux_plane + (long long)r * a.pitch + j] = c.phi;
            add_source_vp<NC>(sa, Av, c.phi, c.P, Fp);
        }
        if (EDGE || YG) {
            const bool grow = YG && (r < 0 || r >= ny);
            if (ghost_col || grow) sv_ghost(k, c, ghost_col ? bvx : (r < 0 ? k.s.bcv[2] : k.s.bcv[3]));
        }
        c.phi = vsum(c.P);  // zeroth moment of P with its sources
        sv_moments(c);
    };
    auto grad_x = [&](int r, const SvCell& c, F2& g2, F2& g3, float& gm) {
        const float ig = (YG && (r < 0 || r >= ny)) ? 0.f : igx;
        const F2 ig2 = f2(ig);
        g2 = (shfl_dn2(c.P.p[2]) - shfl_up2(c.P.p[2])) * ig2;
        g3 = (shfl_up2(c.P.p[3]) - shfl_dn2(c.P.p[3])) * ig2;
        gm = (__shfl_down_sync(0xffffffffu, c.mx, 1) - __shfl_up_sync(0xffffffffu, c.mx, 1)) * ig;
    };
    struct Low {
        F2 q1, q2, q3;
        float ph;
    };
    auto lower = [&](const RowY& w, const SvCell& c, const F2 g2, const F2 g3, const float gm, Low& lo) {
        const F2 gl = f2(-w.gl, w.gl);
        lo.q1 = F2{w.lp} * c.P.p[1];
        lo.q2 = fma2(gl, g2, F2{w.lp} * c.P.p[2]);
        lo.q3 = fma2(gl, g3, F2{w.lp} * c.P.p[3]);
        lo.ph = fmaf(w.l0, c.phi, fmaf(w.hlo, c.my, -w.gl * gm));
    };
    auto yface = [&](const RowY& w, const SvCell& c, const F2 g2, const F2 g3, const float gm, const Low& lo,
                     F2& f1, F2& f2q, F2& f3) {
        const F2 gu = f2(-w.gu, w.gu);
        const F2 b1 = fma2(F2{w.up}, c.P.p[1], lo.q1);
        const F2 b2 = fma2(gu, g2, fma2(F2{w.up}, c.P.p[2], lo.q2));
        const F2 b3 = fma2(gu, g3, fma2(F2{w.up}, c.P.p[3], lo.q3));
        const F2 pb = f2(lo.ph + fmaf(w.u0, c.phi, fmaf(-w.hup, c.my, -w.gu * gm)));
        f1 = fma2(F2{k.a_f2}, b1, hf2(k, 1, pb));
        f2q = fma2(F2{k.a_f2}, b2, hf2(k, 2, pb));
        f3 = fma2(F2{k.a_f2}, b3, hf2(k, 3, pb));
    };

    bool failed = false;
    SvCell c0;
    V9 U0, F, Fp;
    Low lo;
    F2 pm2 = f2(0.f), pm3 = f2(0.f);
    float mym = 0.f, ig0 = 0.f, ry0 = 0.f;
#pragma unroll 1
    for (int r = y0 - 1; r <= y1; ++r) {
        const RowY w = rw[r + 1];
        if (!load_row(r, F)) { failed = true; break; }
        SvCell c;
        F2 g2, g3, f1 = f2(0.f), fq2 = f2(0.f), f3 = f2(0.f);
        float gm;
        cell_row(r, F, c, Fp);
        grad_x(r, c, g2, g3, gm);
        if (r >= y0) yface(w, c, g2, g3, gm, lo, f1, fq2, f3);  // the face below row r
        if (r > y0) {
            // the x-face east of (j, r-1) and the update of row r - 1 (Eqs. 2.19, 2.20, 2.26, 2.22, 2.12)
            const float igy = EDGE ? ig0 * ymask : ig0;
            const F2 igy2 = f2(igy);
            const F2 gy2 = (c.P.p[2] - pm2) * igy2, gy3 = (c.P.p[3] - pm3) * igy2;
            const float gmy = (c.my - mym) * igy;
            const F2 l0 = axLp * c0.P.p[0], r0 = axRp * c0.P.p[0];
            const F2 l2 = fma2(gxL, gy2, axLp * c0.P.p[2]), r2 = fma2(gxR, gy2, axRp * c0.P.p[2]);
            const F2 l3 = fma2(gxL, gy3, axLn * c0.P.p[3]), r3 = fma2(gxR, gy3, axRn * c0.P.p[3]);
            const float pl = fmaf(eL0, c0.phi, fmaf(eLx, c0.mx, eLy * gmy));
            const float pr = fmaf(wR0, c0.phi, fmaf(wRx, c0.mx, wRy * gmy));
            const F2 b0 = l0 + shfl_dn2(r0), b2 = l2 + shfl_dn2(r2), b3 = l3 + shfl_dn2(r3);
            const F2 pb = f2(pl + __shfl_down_sync(0xffffffffu, pr, 1));
            const F2 e0 = fma2(F2{k.a_f2}, b0, hf2(k, 0, pb));
            const F2 e2 = fma2(F2{k.a_f2}, b2, hf2(k, 2, pb));
            const F2 e3 = fma2(F2{k.a_f2}, b3, hf2(k, 3, pb));
            const F2 d0 = e0 - shfl_up2(e0), d2 = e2 - shfl_up2(e2), d3 = e3 - shfl_up2(e3);
            const F2 ryn = sgn2(0.f, -ry0, 1);
            V9 o;
            o.z = U0.z;
            o.p[0] = fma2(rxp, d0, U0.p[0]);
            o.p[1] = fma2(ryn, f1, U0.p[1]);
            o.p[2] = fma2(rxp, d2, fma2(ryn, fq2, U0.p[2]));
            o.p[3] = fma2(rxn, d3, fma2(ryn, f3, U0.p[3]));
            if (updates) {
                float* out = a.fout + (long long)(r - 1) * a.pitch + j;
                out[0] = o.z;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    out[PA(q) * a.plane] = o.p[q].v.x;
                    out[PB(q) * a.plane] = o.p[q].v.y;
                }
            }
            pm2 = c0.P.p[2];
            pm3 = c0.P.p[3];
            mym = c0.my;
        } else if (r < y0) {
            pm2 = c.P.p[2];
            pm3 = c.P.p[3];
            mym = c.my;
        }
        if (r >= y0) {  // row r: ftilde^+ plus the flux of the face below it
            const F2 ryp = sgn2(0.f, w.ry, 1);
            U0 = Fp;
            U0.p[1] = fma2(ryp, f1, U0.p[1]);
            U0.p[2] = fma2(ryp, fq2, U0.p[2]);
            U0.p[3] = fma2(ryp, f3, U0.p[3]);
        }
        lower(w, c, g2, g3, gm, lo);  // the face above row r
        c0 = c;
        ig0 = w.igy;
        ry0 = w.ry;
    }
    if (failed && lane == 0) {
        atomicOr(a.err, 1);
        for (int q = consumed; q < issued; ++q) {
            mbar_wait_bounded(&bars[s], ph, 100000000ull);
            if (++s == S) { s = 0; ph ^= 1u; }
        }
    }
    __syncwarp();
}

#ifndef DUGKS_SV_SRC_MIN_WARPS
#define DUGKS_SV_SRC_MIN_WARPS 16
#endif

// One one-warp CTA per (strip, row segment) with the source terms.
template <int NC>
__global__ void __launch_bounds__(32, DUGKS_SV_SRC_MIN_WARPS)
    step_vp_src(const __grid_constant__ CUtensorMap tin, const StepArgs<float, NC> a, const ConstsP<NC> k,
                const RowY* __restrict__ rw, const SegPlan sp, const int S, const __grid_constant__ SrcArgs<float> sa,
                const __grid_constant__ CUtensorMap taux) {
    using L = WarpLayout<float>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(S) * sa.stage_bytes);
    const int lane = threadIdx.x;
    const int xw = blockIdx.x * L::WI;
    int y0, y1;
    seg_rows_of(sp, int(blockIdx.y), a.ny, y0, y1);
    if (y0 >= a.ny || xw >= a.nx) return;
    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool edge = xw - 1 < 0 || xw + L::WI >= a.nx;
    const bool yg = !a.yper && (y0 == 0 || y1 == a.ny);
    if (!edge && !yg)
        sv_rows_src<NC, true>(&tin, &taux, a, k, rw, sa, smem, bars, S, lane, xw, y0, y1, false, false);
    else
        sv_rows_src<NC>(&tin, &taux, a, k, rw, sa, smem, bars, S, lane, xw, y0, y1, edge, yg);
}

}  // namespace dugks
