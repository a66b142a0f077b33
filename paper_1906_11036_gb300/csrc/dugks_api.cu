// dugks_api.cu -- host side of the C ABI declared in include/dugks.h.
//
// Owns the context (two ftilde buffers, mesh metrics, TMA descriptors, the
// staging and reduction buffers), validates setups, precomputes the
// per-velocity equilibrium polynomials (Eq. 2.3 with B = u b(phi),
// D = d(phi) I, C = u u int_0^phi b'^2, Remark 3) and the relaxation
// coefficients of Eqs. 2.13, 2.21 and 2.22, and launches the kernels.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dugks.h"
#include "dugks_adjoint.cuh"
#include "dugks_adjoint_rows.cuh"
#include "dugks_batch.cuh"
#include "dugks_kernels.cuh"
#include "dugks_step_vp.cuh"

using namespace dugks;

namespace {

constexpr int NC_LARGE = 16;  // up to degree 15 (nb, nd <= 8)

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

struct dugks_ctx {
    int device = 0;
    int nx = 0, ny = 0, precision = 32, kernel = DUGKS_KERNEL_FUSED;
    int xper = 1, yper = 1;
    double bcv[4] = {0, 0, 0, 0};
    double c = 1, dt = 0, lambda = 0, cfl = 0;
    int nc = NC_LARGE;  // equilibrium polynomial coefficients used by the step (3, 4 or 16)
    int nc_u = NC_LARGE;  // the same, large enough for b(phi) and int b'^2 of the u-derivative
    double feq_coef[Q][NC_LARGE];
    double a_bp = 0, b_bp = 0, a_tp = 0, b_tp = 0, a_f = 0, b_f = 0, hc = 0;
    std::vector<double> xf, yf;
    long long pitch = 0, plane = 0;
    size_t elem = 4;
    cudaStream_t stream = nullptr;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    void* fxm = nullptr;  // FaceM<T>[nx+3]
    void* fym = nullptr;  // FaceM<T>[ny+3]
    void* cxm = nullptr;  // CellM<T>[nx+2]
    void* cym = nullptr;  // CellM<T>[ny+2]
    RowY* rowy = nullptr; // FP32: per-row y metrics of step_vp, rows -1 .. ny
    double* dxv = nullptr;  // cell widths (double) for the mass
    double* dyv = nullptr;
    double* staging = nullptr;  // nx*ny doubles for host transfers
    double* partial = nullptr;  // reduction partials
    double* mass_dev = nullptr;
    int* err_dev = nullptr;
    int red_blocks = 0;
    CUtensorMap tmap[2];
    int nt = 32, stages = 8, seg_rows = 0, nstrips = 0, nseg = 0, occupancy = 0;
    int seg_rows_src = 0, nseg_src = 0;  // row segments of the source-term kernel (FP64: uniform)
    SegPlan sp_src{0, 0, 0};              // the FP32 source-term kernel's segment plan
    bool plain = false;                   // step_vp with the interior variant (long-segment plans)
    int nseg_sp_src = 0;
    SegPlan sp{1, 0, 1};  // step_vp: long segments first, then short ones
    long long steps_done = 0;
    // adjoint work buffers (allocated on first use)
    void* adj_ax = nullptr;
    void* adj_ay = nullptr;
    double* adj_partial = nullptr;  // 3 adj_partials(): dJ/dlambda, dJ/du_x, dJ/du_y per block
    double* adj_upart = nullptr;    // 3 x kInitBlocks: the initialisation's u partials
    int adj_used = 0;               // partial slots the last adjoint launch wrote (the sums read these)
    void* adj_ws = nullptr;         // dugks_adjoint's states (checkpoints, a segment, two lambdas), kept
    size_t adj_ws_bytes = 0;        //   for later calls and grown when a call needs more
    double* adj_dalpha = nullptr;
    // source terms (dugks_set_source)
    double ux = 0, uy = 0;
    int nb = 0;
    double bcoef[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int c_zero = 0;
    int nsrc = 0;
    double src_rate[8];
    int src_power[8];
    void* src_field = nullptr;            // S_k [nsrc][ny][nx], precision's type
    void* hist[2] = {nullptr, nullptr};   // phi^{n-1} (read) / phi^n (written), alternating with cur
    // FP32 velocity-pair path: fields and history as nsrc + 1 pitched planes, alternating with cur,
    // staged by TMA into the same ring stage as ftilde
    void* aux[2] = {nullptr, nullptr};
    CUtensorMap taux[2];
    int aux_box = 0, src_stage = 0;  // bytes of one aux box; bytes of one ring stage
    bool src_first = true;
    double t = 0, t0 = 0;   // time of the state; source start time
    double tbase = 0;       // t = tbase + tsteps * dt (tbase set by set_source, init_phi, load_state)
    long long tsteps = 0;
    int adj_kernel = DUGKS_ADJ_AUTO;  // dugks_set_adjoint_kernel
    int feq_check = 0;                // dugks_set_feq_check: initialisations test the equilibrium
    std::string last_error;
};

constexpr int kBatchShortRows = 8;       // rows of the short tiles at the end of the batched queue

struct dugks_batch {
    int n = 0, device = 0, nc = 3;
    std::vector<dugks_ctx*> ctx;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* d_insts = nullptr;   // BatchInst<nc>[n]
    BatchTile* d_tiles = nullptr;  // the tile queue
    bool split = true;             // long segments, then short tiles at the end of the queue
    double long_frac = 0.8;        // with split: share of an instance's rows in long tiles
    int* d_counters = nullptr;  // one per launch of a graph (plus the remainder)
    int* d_err = nullptr;
    int ntiles = 0, seg_target = 48, blocks = 0, stages = 4;
    static constexpr int kGraphSteps = 50;  // even: a replay leaves the parity unchanged
    cudaGraphExec_t graph = nullptr;
    int parity = 0;
    long long steps_done = 0;
    std::string last_error;
};

namespace {

dugks_status cuda_fail(dugks_ctx* ctx, cudaError_t e, const char* what) {
    if (ctx) {
        ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return e == cudaErrorMemoryAllocation ? DUGKS_ERR_NOMEM : DUGKS_ERR_CUDA;
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
    } while (0)

bool finite_all(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// int_0^phi b'(s)^2 ds as polynomial coefficients: sum_{k,l>=1} k l b_k b_l phi^{k+l-1}/(k+l-1)
void aux_moment_poly(const dugks_coef* cf, double* out /* NC_LARGE */) {
    for (int m = 0; m < NC_LARGE; ++m) out[m] = 0.0;
    if (cf->c_zero) return;
    for (int k = 1; k < cf->nb; ++k)
        for (int l = 1; l < cf->nb; ++l) {
            const int m = k + l - 1;
            out[m] += double(k) * double(l) * cf->b[k] * cf->b[l] / double(m);
        }
}

// Equilibrium (Eq. 2.3) per velocity as a polynomial in phi, coefficients
// out[i][m] of phi^m, with e_i the unit direction and c_s^2 = c^2/3:
//   feq_i = w_i [ phi + 3 (e_i.u)/c b + (3|e_i|^2 - 2)/2 (d - phi)
//                 + (9 (e_i.u)^2 - 3 |u|^2) / (2 c^2) Cint ]
// A tensor D adds D:(e_i e_i c^2 - c_s^2 I)/(2 c_s^2) = [(3 ex^2 - 1) dxx + 6 ex ey dxy + (3 ey^2 - 1) dyy]/2
// in place of (3|e_i|^2 - 2)/2 d; the -phi part keeps the isotropic form.  *maxdeg: highest
// degree with a nonzero coefficient (at least 1).
void feq_coefficients(const dugks_vset* vset, const dugks_coef* coef, double (*out)[NC_LARGE], int* maxdeg) {
    double cint[NC_LARGE];
    aux_moment_poly(coef, cint);
    const double wts[Q] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const double ux = coef->u[0], uy = coef->u[1], c = vset->c;
    *maxdeg = 1;
    for (int i = 0; i < Q; ++i) {
        const double eu = EX(i) * ux + EY(i) * uy;
        const double e2 = double(EX(i) * EX(i) + EY(i) * EY(i));
        const double kb = 3.0 * eu / c, kd = (3.0 * e2 - 2.0) / 2.0;
        const double kxx = (3.0 * EX(i) * EX(i) - 1.0) / 2.0, kyy = (3.0 * EY(i) * EY(i) - 1.0) / 2.0;
        const double kxy = 3.0 * EX(i) * EY(i);
        const double kc = (9.0 * eu * eu - 3.0 * (ux * ux + uy * uy)) / (2.0 * c * c);
        for (int m = 0; m < NC_LARGE; ++m) {
            const double bm = m < coef->nb ? coef->b[m] : 0.0;
            const double one = m == 1 ? 1.0 : 0.0;
            double dpart;
            if (coef->d_tensor) {
                const double xx = m < coef->ndt ? coef->dxx[m] : 0.0, xy = m < coef->ndt ? coef->dxy[m] : 0.0;
                const double yy = m < coef->ndt ? coef->dyy[m] : 0.0;
                dpart = kxx * xx + kxy * xy + kyy * yy - kd * one;
            } else {
                const double dm = m < coef->nd ? coef->d[m] : 0.0;
                dpart = kd * (dm - one);
            }
            const double v = wts[i] * (one + kb * bm + dpart + kc * cint[m]);
            out[i][m] = v;
            if (v != 0.0) *maxdeg = std::max(*maxdeg, m);
        }
    }
}

double poly_eval(const double* c, int n, double x) {
    double s = c[n - 1];
    for (int m = n - 2; m >= 0; --m) s = s * x + c[m];
    return s;
}

// Positivity of the equilibrium over phi in [lo, hi] (the rest velocity as phi minus the
// sum of the others, as the kernels form it).  *feq_min: the smallest f^eq_i(phi); return
// value: the smallest margin min_i f^eq_i(phi) + kFeqTol max_i |f^eq_i(phi)|, negative when
// some equilibrium is negative by more than kFeqTol of the largest one at the same phi.
// 4097 samples per velocity, then a golden-section refinement around the smallest sample.
constexpr double kFeqTol = 1e-3;
double feq_margin_over(const double (*cf)[NC_LARGE], double lo, double hi, double* feq_min) {
    auto eval = [&](double x, double& mn) {
        double v[Q], s = 0.0;
        for (int q = 1; q < Q; ++q) {
            v[q] = poly_eval(cf[q], NC_LARGE, x);
            s += v[q];
        }
        v[0] = x - s;
        double mx = 0.0;
        mn = INFINITY;
        for (int q = 0; q < Q; ++q) {
            mn = std::min(mn, v[q]);
            mx = std::max(mx, std::fabs(v[q]));
        }
        return mn + kFeqTol * mx;
    };
    const int N = 4096;
    double best = INFINITY, fmin = INFINITY, mn;
    int kbest = 0;
    for (int k = 0; k <= N; ++k) {
        const double g = eval(lo + (hi - lo) * double(k) / N, mn);
        fmin = std::min(fmin, mn);
        if (g < best) { best = g; kbest = k; }
    }
    double a = lo + (hi - lo) * double(std::max(kbest - 1, 0)) / N;
    double b = lo + (hi - lo) * double(std::min(kbest + 1, N)) / N;
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    for (int it = 0; it < 60 && b > a; ++it) {
        const double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
        double m1, m2;
        if (eval(x1, m1) < eval(x2, m2)) b = x2; else a = x1;
        fmin = std::min(fmin, std::min(m1, m2));
    }
    best = std::min(best, eval(0.5 * (a + b), mn));
    fmin = std::min(fmin, mn);
    if (feq_min) *feq_min = fmin;
    return best;
}

template <typename T>
void build_metrics(const std::vector<double>& f, bool per, double hcv, double dt, double c, std::vector<FaceM<T>>& fm,
                   std::vector<CellM<T>>& cm, std::vector<double>& width) {
    const int n = int(f.size()) - 1;
    std::vector<double> xc(n + 2);  // centres j = -1..n at index j+1
    for (int j = 0; j < n; ++j) xc[j + 1] = 0.5 * (f[j] + f[j + 1]);
    const double L = f[n] - f[0];
    if (per) {
        xc[0] = xc[n] - L;
        xc[n + 1] = xc[1] + L;
    } else {  // mirror images across the walls
        xc[0] = 2.0 * f[0] - xc[1];
        xc[n + 1] = 2.0 * f[n] - xc[n];
    }
    fm.assign(n + 3, FaceM<T>{T(0.5), T(0), T(0), T(0)});
    for (int q = 0; q <= n; ++q) {  // face q between columns q-1 and q
        const double xl = xc[q], xr = xc[q + 1];
        const double dxc = xr - xl, w = (f[q] - xl) / dxc;
        double tl = 1.0 - w, tr = w;
        if (!per && q == 0) { tl = 0.0; tr = 1.0; }
        if (!per && q == n) { tl = 1.0; tr = 0.0; }
        fm[q + 1] = FaceM<T>{T(w), T(hcv / dxc), T(tl), T(tr)};
    }
    cm.assign(n + 2, CellM<T>{T(0), T(0)});
    width.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        cm[j + 1] = CellM<T>{T(1.0 / (xc[j + 2] - xc[j])), T(dt * c / (f[j + 1] - f[j]))};
        width[j] = f[j + 1] - f[j];
    }
}

// Weights (a, b) of a convex-type combination a f + b feq with a + b = 1 exactly in T.
// a lies in (-1, 1) for Eqs. 2.13 and 2.21, so b = 1 - a is in (0, 2); with b rounded
// first, 1 - b is exact (Sterbenz) and a + b == 1 in T: rounded weights cannot bias
// the discrete mass.
template <typename T>
void unit_pair(double a_exact, T& a, T& b) {
    b = T(1.0 - double(T(a_exact)));
    a = T(1.0 - double(b));
}

template <typename T, int NC>
Consts<T, NC> make_consts(const dugks_ctx* ctx) {
    Consts<T, NC> k;
    for (int i = 0; i < Q; ++i)
        for (int m = 0; m < NC; ++m) k.feq[i][m] = T(ctx->feq_coef[i][m]);
    // Eq. 2.21 weights also sum to one (2h = dt)
    unit_pair<T>(ctx->a_bp, k.a_bp, k.b_bp);
    // Eq. 2.13 weights sum to one; keep that exact in the stored precision
    unit_pair<T>(ctx->a_tp, k.a_tp, k.b_tp);
    k.a_f = T(ctx->a_f); k.b_f = T(ctx->b_f);
    for (int i = 0; i < Q; ++i)
        for (int m = 0; m < NC; ++m) {
            k.hbp[i][m] = T(double(k.b_bp) * ctx->feq_coef[i][m]);
            k.hf[i][m] = T(ctx->b_f * ctx->feq_coef[i][m]);
        }
    k.third = T(1.0 / 3.0);
    k.hc = T(ctx->hc);
    for (int w = 0; w < 4; ++w) k.bcv[w] = T(ctx->bcv[w]);
    return k;
}

template <int NC>
ConstsP<NC> make_constsp(const dugks_ctx* ctx) {
    ConstsP<NC> k;
    k.s = make_consts<float, NC>(ctx);
    for (int q = 0; q < 4; ++q)
        for (int m = 0; m < NC; ++m) {
            k.hbp[q][m] = make_float2(k.s.hbp[PA(q)][m], k.s.hbp[PB(q)][m]);
            k.hf[q][m] = make_float2(k.s.hf[PA(q)][m], k.s.hf[PB(q)][m]);
        }
    k.a_bp = k.s.a_bp; k.b_bp = k.s.b_bp; k.third = k.s.third; k.hc = k.s.hc;
    k.a_bp2 = make_float2(k.a_bp, k.a_bp);
    k.a_f2 = make_float2(k.s.a_f, k.s.a_f);
    k.third2 = make_float2(k.third, k.third);
    return k;
}

template <typename T, int NC>
StepArgs<T, NC> make_args(const dugks_ctx* ctx, int from) {
    StepArgs<T, NC> a;
    a.fin = static_cast<const T*>(ctx->buf[from]);
    a.fout = static_cast<T*>(ctx->buf[1 - from]);
    a.nx = ctx->nx; a.ny = ctx->ny;
    a.pitch = ctx->pitch; a.plane = ctx->plane;
    a.xper = ctx->xper; a.yper = ctx->yper;
    a.fx = static_cast<const FaceM<T>*>(ctx->fxm);
    a.fy = static_cast<const FaceM<T>*>(ctx->fym);
    a.cx = static_cast<const CellM<T>*>(ctx->cxm);
    a.cy = static_cast<const CellM<T>*>(ctx->cym);
    a.err = ctx->err_dev;
    return a;
}

void* fused_fn(const dugks_ctx* ctx) {
    if (ctx->precision == 32) {
        switch (ctx->nc) {
            case 3: return ctx->plain ? reinterpret_cast<void*>(&step_vp<3, true>) : reinterpret_cast<void*>(&step_vp<3, false>);
            case 4: return ctx->plain ? reinterpret_cast<void*>(&step_vp<4, true>) : reinterpret_cast<void*>(&step_vp<4, false>);
            default: return reinterpret_cast<void*>(&fused_step<float, NC_LARGE>);  // high degree: scalar path
        }
    }
    switch (ctx->nc) {
        case 3: return reinterpret_cast<void*>(&fused_step<double, 3>);
        case 4: return reinterpret_cast<void*>(&fused_step<double, 4>);
        default: return reinterpret_cast<void*>(&fused_step<double, NC_LARGE>);
    }
}

// the FP32 velocity-pair kernel takes the source fields from the TMA-staged aux planes
bool src_uses_aux(const dugks_ctx* ctx) { return ctx->precision == 32 && ctx->nc != NC_LARGE; }

size_t src_vp_smem(const dugks_ctx* ctx) { return size_t(ctx->stages) * (ctx->src_stage + 8) + 128; }

size_t fused_smem(const dugks_ctx* ctx) {
    return ctx->precision == 32 ? WarpLayout<float>::bytes(ctx->stages) : WarpLayout<double>::bytes(ctx->stages);
}

EncodeTiledFn tiled_encoder(dugks_ctx* ctx) {
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            ctx->last_error = "cuTensorMapEncodeTiled is not available from the driver";
            return nullptr;
        }
        encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    return encode;
}

dugks_status make_tensor_maps(dugks_ctx* ctx) {
    EncodeTiledFn encode = tiled_encoder(ctx);
    if (!encode) return DUGKS_ERR_CUDA;
    const int align = 16 / int(ctx->elem);
    const cuuint64_t dims[3] = {cuuint64_t(ctx->nx), cuuint64_t(ctx->ny), cuuint64_t(Q)};
    const cuuint64_t strides[2] = {cuuint64_t(ctx->pitch) * ctx->elem, cuuint64_t(ctx->plane) * ctx->elem};
    const cuuint32_t box[3] = {cuuint32_t(ctx->precision == 32 ? WarpLayout<float>::BOXW : WarpLayout<double>::BOXW),
                               1u, cuuint32_t(Q)};
    (void)align;
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    for (int b = 0; b < 2; ++b) {
        CUresult r = encode(&ctx->tmap[b], ctx->precision == 32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                            3, ctx->buf[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            char buf[128];
            snprintf(buf, sizeof(buf), "cuTensorMapEncodeTiled failed (%d)", int(r));
            ctx->last_error = buf;
            return DUGKS_ERR_CUDA;
        }
    }
    return DUGKS_OK;
}

// step_vp's segments: every strip gets K = slots / nstrips long segments that together
// cover about a fraction `first` of its rows (one wave of warps), then short segments of
// seg_short rows.  Blocks start in launch order, so the short segments fill in behind
// the long ones as warps finish, and each warp pays the pipeline fill (two extra rows
// and the latency of its first loads) over a long segment.  Grids without enough rows
// for that keep the uniform plan.
#ifndef DUGKS_PLAN_FIRST
#define DUGKS_PLAN_FIRST 0.8
#endif
#ifndef DUGKS_PLAN_SHORT
#define DUGKS_PLAN_SHORT 8
#endif
// 2048^2 (us per step): 0.8 / 8 rows 65.9, 0.85 / 8 65.6, 0.9 / 8 66.2, 0.8 / 6 66.6, 0.9 / 6 65.9,
// 0.9 / 10 66.4, 0.95 / 8 68.0
constexpr double kPlanFirst = DUGKS_PLAN_FIRST;  // share of the rows in the first wave of long segments
constexpr int kPlanShort = DUGKS_PLAN_SHORT;      // rows of the short segments after them
#ifndef DUGKS_SRC_PLAN_FIRST
#define DUGKS_SRC_PLAN_FIRST 0.7
#endif
#ifndef DUGKS_SRC_PLAN_SHORT
#define DUGKS_SRC_PLAN_SHORT 8
#endif
// the same for the source-term kernel, from its own occupancy (Example 4.5 at 2048^2, us per
// step: uniform 20-row segments 131.8; long share 0.9 141.0, 0.8 132.7, 0.7 121.8, 0.65 122.2,
// 0.6 123.3, 0.5 125.4 with 8-row short segments; 0.8 with 12 or 16 rows 132.5, 131.7)
constexpr double kSrcPlanFirst = DUGKS_SRC_PLAN_FIRST;
constexpr int kSrcPlanShort = DUGKS_SRC_PLAN_SHORT;
// Long segments over the first wave (share `first` of the rows), short ones after them;
// false (and nothing set) where the grid has too few rows for it.
bool plan_long_short(const dugks_ctx* ctx, long long slots, double first, int seg_short, SegPlan& sp, int& nseg) {
    const long long K = std::max<long long>(1, slots / ctx->nstrips);
    const int L = int(first * ctx->ny / double(K));
    if (L < 2 * seg_short || L < 24) return false;
    const int rest = ctx->ny - int(K) * L;
    if (rest <= 0) return false;
    const int nshort = (rest + seg_short - 1) / seg_short;
    sp = SegPlan{L, int(K), seg_short};
    nseg = int(K) + nshort;
    return true;
}

// Strip and segment counts of the fused kernels for this grid: one warp per
// (30-column strip, row segment), at least 16 rows per segment so that the two
// pipeline-fill rows stay cheap; about three waves of segments, which the block
// scheduler balances.  The FP32 step (step_vp) then takes the long-then-short
// plan where the grid has the rows for it (2048^2: 35 segments of 46 rows per
// strip, then 8-row segments; 66.5 us against 70.0 us for uniform 20-row ones).
dugks_status plan_fused(dugks_ctx* ctx) {
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaDeviceGetAttribute");
    ctx->nt = 32;
    ctx->stages = 3;  // rows in flight per warp
    void* fn = fused_fn(ctx);
    const size_t smem = fused_smem(ctx);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (occ < 1) {
        ctx->last_error = "fused kernel does not fit on an SM";
        return DUGKS_ERR_UNSUPPORTED;
    }
    ctx->occupancy = occ;
    const int wi = WarpLayout<float>::WI;
    ctx->nstrips = (ctx->nx + wi - 1) / wi;
    const long long slots = (long long)sms * occ;
    const long long max_seg = std::max(1, ctx->ny / 16);
    auto cut = [&](long long nseg, int& seg_rows, int& nseg_out) {
        nseg = std::max<long long>(1, std::min<long long>(nseg, max_seg));
        seg_rows = int((ctx->ny + nseg - 1) / nseg);
        nseg_out = (ctx->ny + seg_rows - 1) / seg_rows;
    };
    cut(3 * slots / ctx->nstrips, ctx->seg_rows, ctx->nseg);
    cut(3 * slots / ctx->nstrips, ctx->seg_rows_src, ctx->nseg_src);
    ctx->sp = SegPlan{ctx->seg_rows, ctx->nseg, ctx->seg_rows};
    ctx->plain = false;
    if (ctx->precision == 32 && ctx->nc != NC_LARGE && plan_long_short(ctx, slots, kPlanFirst, kPlanShort, ctx->sp, ctx->nseg)) {
        ctx->seg_rows = ctx->sp.seg_long;
        ctx->plain = true;  // the interior variant pays on long segments (step_vp)
        e = cudaFuncSetAttribute(fused_fn(ctx), cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
    ctx->sp_src = SegPlan{ctx->seg_rows_src, ctx->nseg_src, ctx->seg_rows_src};
    ctx->nseg_sp_src = ctx->nseg_src;
    return DUGKS_OK;
}

// Per-row y metrics of step_vp (rows -1 .. ny at index k + 1) from the y-face and
// y-cell metrics: the reconstruction weights of the faces below and above each row
// (Eqs. 2.19, 2.20), its central-difference factor and its flux factor (Eq. 2.12).
std::vector<RowY> make_rowy(const std::vector<FaceM<float>>& fy, const std::vector<CellM<float>>& cy, int ny,
                            float hc) {
    std::vector<RowY> rw(size_t(ny) + 2);
    for (int k = -1; k <= ny; ++k) {
        const FaceM<float> b = fy[size_t(k) + 1], t = fy[size_t(k) + 2];
        RowY r;
        r.up = make_float2(b.w - b.hcd, b.w + b.hcd);
        r.u0 = b.w;
        r.gu = hc * b.tr;
        r.lp = make_float2((1.f - t.w) + t.hcd, (1.f - t.w) - t.hcd);
        r.l0 = 1.f - t.w;
        r.gl = hc * t.tl;
        r.igy = cy[size_t(k) + 1].ig;
        r.ry = cy[size_t(k) + 1].r;
        r.hup = b.hcd;
        r.hlo = t.hcd;
        rw[size_t(k) + 1] = r;
    }
    return rw;
}

// Launch arguments of the source terms for the step from ctx->t (Eqs. 2.3, 2.12, 2.18).
template <typename T>
SrcArgs<T> make_src_args(const dugks_ctx* ctx) {
    SrcArgs<T> sa{};
    sa.nterms = ctx->nsrc;
    sa.first = ctx->src_first ? 1 : 0;
    for (int q = 0; q < ctx->nsrc; ++q) {
        sa.power[q] = ctx->src_power[q];
        sa.dpow[q] = ctx->src_power[q] - (q ? ctx->src_power[q - 1] : 0);
        sa.en[q] = T(std::exp(ctx->src_rate[q] * ctx->t));
        sa.ep[q] = ctx->src_first ? sa.en[q] : T(std::exp(ctx->src_rate[q] * (ctx->t - ctx->dt)));
    }
    sa.ndb = std::max(0, ctx->nb - 1);  // b'(phi) = sum_m (m+1) b_{m+1} phi^m
    for (int m = 0; m + 1 < ctx->nb; ++m) sa.db[m] = T(double(m + 1) * ctx->bcoef[m + 1]);
    const double cs2 = ctx->c * ctx->c / 3.0, h = 0.5 * ctx->dt, lam = ctx->lambda;
    const double wr = 2.0 * lam * h / (2.0 * lam + h);  // weight of R in Eq. 2.18
    const double wts[Q] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    for (int i = 0; i < Q; ++i) {
        const double cu = ctx->c * (EX(i) * ctx->ux + EY(i) * ctx->uy) / cs2;  // c_i.u / c_s^2
        sa.kP_g[i] = T(wr * wts[i] * cu);
        sa.kP_f[i] = T(h * wts[i]);
        sa.kU_g[i] = T(ctx->dt * wts[i] * cu);
        sa.kU_f[i] = T(ctx->dt * wts[i]);
    }
    sa.field = static_cast<const T*>(ctx->src_field);
    sa.fplane = (long long)ctx->nx * ctx->ny;
    sa.hin = static_cast<const T*>(ctx->hist[ctx->cur]);
    sa.hout = static_cast<T*>(ctx->hist[ctx->cur ^ 1]);
    sa.aux_in = static_cast<const T*>(ctx->aux[ctx->cur]);
    sa.aux_out = static_cast<T*>(ctx->aux[ctx->cur ^ 1]);
    sa.aux_plane = ctx->plane;
    sa.aux_box = ctx->aux_box;
    sa.stage_bytes = ctx->src_stage;
    return sa;
}

template <typename T, int NC>
cudaError_t launch_step(dugks_ctx* ctx) {
    const StepArgs<T, NC> a = make_args<T, NC>(ctx, ctx->cur);
    const Consts<T, NC> k = make_consts<T, NC>(ctx);
    if (ctx->nsrc > 0) {  // the fused kernel with the source terms: velocity pairs in FP32, else scalar
        dim3 grid(ctx->nstrips, ctx->nseg_src);
        if constexpr (sizeof(T) == 4 && NC != NC_LARGE)
            step_vp_src<NC><<<dim3(ctx->nstrips, ctx->nseg_sp_src), 32, src_vp_smem(ctx), ctx->stream>>>(
                ctx->tmap[ctx->cur], a, make_constsp<NC>(ctx), ctx->rowy, ctx->sp_src, ctx->stages,
                make_src_args<float>(ctx), ctx->taux[ctx->cur]);
        else
            fused_step_src<T, NC><<<grid, 32, fused_smem(ctx), ctx->stream>>>(ctx->tmap[ctx->cur], a, k,
                                                                             ctx->seg_rows_src, ctx->stages,
                                                                             make_src_args<T>(ctx));
        return cudaGetLastError();
    }
    if (ctx->kernel == DUGKS_KERNEL_NAIVE) {
        dim3 grid((ctx->nx + 127) / 128, std::min(ctx->ny, 65535));
        naive_step<T, NC><<<grid, 128, 0, ctx->stream>>>(a, k);
    } else {
        dim3 grid(ctx->nstrips, ctx->nseg);
        if constexpr (sizeof(T) == 4 && NC != NC_LARGE)
            if (ctx->plain)
                step_vp<NC, true><<<grid, 32, fused_smem(ctx), ctx->stream>>>(
                    ctx->tmap[ctx->cur], a, make_constsp<NC>(ctx), ctx->rowy, ctx->sp, ctx->stages);
            else
                step_vp<NC, false><<<grid, 32, fused_smem(ctx), ctx->stream>>>(
                    ctx->tmap[ctx->cur], a, make_constsp<NC>(ctx), ctx->rowy, ctx->sp, ctx->stages);
        else
            fused_step<T, NC><<<grid, 32, fused_smem(ctx), ctx->stream>>>(ctx->tmap[ctx->cur], a, k, ctx->seg_rows,
                                                                         ctx->stages);
    }
    return cudaGetLastError();
}

cudaError_t launch_step_any(dugks_ctx* ctx) {
    if (ctx->precision == 32) {
        switch (ctx->nc) {
            case 3: return launch_step<float, 3>(ctx);
            case 4: return launch_step<float, 4>(ctx);
            default: return launch_step<float, NC_LARGE>(ctx);
        }
    }
    switch (ctx->nc) {
        case 3: return launch_step<double, 3>(ctx);
        case 4: return launch_step<double, 4>(ctx);
        default: return launch_step<double, NC_LARGE>(ctx);
    }
}

template <typename T, typename Tin>
cudaError_t launch_init(dugks_ctx* ctx, const Tin* phi0) {
    const long long n = (long long)ctx->nx * ctx->ny;
    const int blocks = int(std::min<long long>((n + 255) / 256, 65535));
    T* f = static_cast<T*>(ctx->buf[ctx->cur]);
    // the initialisation is not on the hot path: always the generic polynomial degree
    init_kernel<T, NC_LARGE, Tin><<<blocks, 256, 0, ctx->stream>>>(phi0, f, ctx->nx, ctx->ny, ctx->pitch, ctx->plane,
                                                                  make_consts<T, NC_LARGE>(ctx),
                                                                  ctx->feq_check ? ctx->err_dev : nullptr);
    return cudaGetLastError();
}

template <typename T, typename Tout>
cudaError_t launch_phi(dugks_ctx* ctx, Tout* phi) {
    const T* f = static_cast<const T*>(ctx->buf[ctx->cur]);
    phi_mass_kernel<T, Tout><<<ctx->red_blocks, 256, 0, ctx->stream>>>(f, phi, ctx->nx, ctx->ny, ctx->pitch, ctx->plane,
                                                                       ctx->dxv, ctx->dyv, ctx->partial);
    sum_partials_kernel<<<1, 256, 0, ctx->stream>>>(ctx->partial, ctx->red_blocks, ctx->mass_dev);
    return cudaGetLastError();
}

void free_ctx(dugks_ctx* ctx) {
    if (!ctx) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    for (void* p : {ctx->buf[0], ctx->buf[1], ctx->fxm, ctx->fym, ctx->cxm, ctx->cym, static_cast<void*>(ctx->rowy),
                    ctx->adj_ax, ctx->adj_ay,
                    ctx->src_field, ctx->hist[0], ctx->hist[1], ctx->aux[0], ctx->aux[1],
                    static_cast<void*>(ctx->adj_partial), static_cast<void*>(ctx->adj_dalpha),
                    static_cast<void*>(ctx->adj_upart), ctx->adj_ws})
        if (p) cudaFree(p);
    for (void* p : {static_cast<void*>(ctx->dxv), static_cast<void*>(ctx->dyv), static_cast<void*>(ctx->staging),
                    static_cast<void*>(ctx->partial), static_cast<void*>(ctx->mass_dev),
                    static_cast<void*>(ctx->err_dev)})
        if (p) cudaFree(p);
    if (prev >= 0) cudaSetDevice(prev);
    delete ctx;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

template <typename T, int NC>
AdjConsts<T, NC> make_adj_consts(const dugks_ctx* ctx) {
    AdjConsts<T, NC> ka;
    for (int i = 0; i < Q; ++i)
        for (int m = 0; m < NC; ++m) ka.dfeq[i][m] = T(m + 1 < NC_LARGE ? double(m + 1) * ctx->feq_coef[i][m + 1] : 0.0);
    const double lam = ctx->lambda, dt = ctx->dt, h = 0.5 * dt;
    const double d1 = 2.0 * lam + dt, d2 = 2.0 * lam + h;
    ka.a_bp = T(ctx->a_bp); ka.b_bp = T(ctx->b_bp);
    ka.a_tp = T(ctx->a_tp); ka.b_tp = T(ctx->b_tp);
    ka.a_f = T(ctx->a_f); ka.b_f = T(ctx->b_f);
    ka.da_bp = T(2.0 * (dt + h) / (d1 * d1)); ka.db_bp = T(-6.0 * h / (d1 * d1));  // d/dlambda of Eq. 2.21 weights
    ka.da_tp = T(4.0 * dt / (d1 * d1)); ka.db_tp = T(-4.0 * dt / (d1 * d1));        // Eq. 2.13
    ka.da_f = T(2.0 * h / (d2 * d2)); ka.db_f = T(-2.0 * h / (d2 * d2));            // Eq. 2.22
    // d feq_i / d u_a = A_ia b(phi) + B_ia Cint(phi) (Eq. 2.3 with B = u b, C = u u Cint, Remark 3)
    double cint[NC_LARGE] = {};
    if (!ctx->c_zero)
        for (int kk = 1; kk < ctx->nb; ++kk)
            for (int l = 1; l < ctx->nb; ++l) {
                const int m = kk + l - 1;
                cint[m] += double(kk) * double(l) * ctx->bcoef[kk] * ctx->bcoef[l] / double(m);
            }
    for (int m = 0; m < NC; ++m) {
        ka.bpoly[m] = T(m < ctx->nb ? ctx->bcoef[m] : 0.0);
        ka.cpoly[m] = T(cint[m]);
    }
    const double wts[Q] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const double c = ctx->c, u[2] = {ctx->ux, ctx->uy};
    for (int i = 0; i < Q; ++i) {
        const double e[2] = {double(EX(i)), double(EY(i))}, eu = e[0] * u[0] + e[1] * u[1];
        for (int ax = 0; ax < 2; ++ax) {
            ka.Au[ax][i] = T(3.0 * wts[i] * e[ax] / c);
            ka.Bu[ax][i] = T(ctx->c_zero ? 0.0 : wts[i] * (9.0 * e[ax] * eu - 3.0 * u[ax]) / (c * c));
        }
    }
    return ka;
}

// the FP32 adjoint's constants on velocity pairs, from the scalar ones
template <int NC>
AdjConstsP<NC> make_adj_consts_p(const dugks_ctx* ctx) {
    const Consts<float, NC> k = make_consts<float, NC>(ctx);
    const AdjConsts<float, NC> ka = make_adj_consts<float, NC>(ctx);
    AdjConstsP<NC> p;
    for (int q = 0; q < 4; ++q) {
        for (int m = 0; m < NC; ++m) {
            p.hbp[q][m] = make_float2(k.hbp[PA(q)][m], k.hbp[PB(q)][m]);
            p.fq[q][m] = make_float2(k.feq[PA(q)][m], k.feq[PB(q)][m]);
            p.dq[q][m] = make_float2(ka.dfeq[PA(q)][m], ka.dfeq[PB(q)][m]);
        }
        for (int ax = 0; ax < 2; ++ax) {
            p.Au[ax][q] = make_float2(ka.Au[ax][PA(q)], ka.Au[ax][PB(q)]);
            p.Bu[ax][q] = make_float2(ka.Bu[ax][PA(q)], ka.Bu[ax][PB(q)]);
        }
    }
    for (int ax = 0; ax < 2; ++ax) {
        p.Au0[ax] = ka.Au[ax][0];
        p.Bu0[ax] = ka.Bu[ax][0];
    }
    for (int m = 0; m < NC; ++m) {
        p.bpoly[m] = ka.bpoly[m];
        p.cpoly[m] = ka.cpoly[m];
    }
    p.a_bp = ka.a_bp; p.b_bp = ka.b_bp; p.a_tp = ka.a_tp; p.b_tp = ka.b_tp; p.a_f = ka.a_f; p.b_f = ka.b_f;
    p.da_bp = ka.da_bp; p.db_bp = ka.db_bp; p.da_tp = ka.da_tp; p.db_tp = ka.db_tp;
    p.da_f = ka.da_f; p.db_f = ka.db_f;
    p.hc = k.hc;
    for (int w = 0; w < 4; ++w) p.bcv[w] = k.bcv[w];
    return p;
}

// adjoint: tiles of kAdjTX x kAdjTY cells (adj_tile_kernel); the wall fold uses 128-thread blocks
constexpr int kAdjThreads = 128;
constexpr int kAdjTX = 32, kAdjTY = 8;
dim3 adj_tile_grid(const dugks_ctx* ctx) {
    return dim3(unsigned((ctx->nx + kAdjTX - 1) / kAdjTX), unsigned((ctx->ny + kAdjTY - 1) / kAdjTY), 1u);
}
int adj_tile_blocks(const dugks_ctx* ctx) {
    const dim3 d = adj_tile_grid(ctx);
    return int(d.x * d.y);
}
// cells next to a Dirichlet wall (adj_wall_kernel), each counted once
long long adj_wall_cells(const dugks_ctx* ctx) {
    const long long nx = ctx->nx, ny = ctx->ny;
    const bool xper = ctx->xper, yper = ctx->yper;
    const long long nrc = yper ? 0 : (ny > 1 ? 2 : 1) * nx;
    const long long nr = yper ? ny : std::max<long long>(0, ny - 2);
    const long long ncc = xper ? 0 : (nx > 1 ? 2 : 1) * nr;
    return nrc + ncc;
}
int adj_wall_blocks(const dugks_ctx* ctx) { return int((adj_wall_cells(ctx) + kAdjThreads - 1) / kAdjThreads); }
int adj_partials(const dugks_ctx* ctx) { return adj_tile_blocks(ctx) + adj_wall_blocks(ctx); }
// blocks of init_adjoint_kernel
int init_blocks(const dugks_ctx* ctx) {
    return int(std::min<long long>(((long long)ctx->nx * ctx->ny + 255) / 256, 65535));
}

dugks_status adj_alloc(dugks_ctx* ctx) {
    if (adj_tile_grid(ctx).y > 65535u) {
        ctx->last_error = "the adjoint supports ny <= 524280";
        return DUGKS_ERR_UNSUPPORTED;
    }
    if (ctx->adj_ax) return DUGKS_OK;
    cudaError_t e;
    const size_t nxf = size_t(ctx->nx + 1) * ctx->ny, nyf = size_t(ctx->nx) * (ctx->ny + 1);
    if ((e = cudaMalloc(&ctx->adj_ax, Q * nxf * ctx->elem)) != cudaSuccess ||
        (e = cudaMalloc(&ctx->adj_ay, Q * nyf * ctx->elem)) != cudaSuccess ||
        (e = cudaMalloc(&ctx->adj_partial, 3 * sizeof(double) * size_t(adj_partials(ctx)))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->adj_dalpha, 3 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->adj_upart, 3 * sizeof(double) * size_t(init_blocks(ctx)))) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc(adjoint buffers)");
    return DUGKS_OK;
}


// *dj_dalpha += (sum of the lambda partials) / c_s^2; dj_du[a] += sum of the u_a partials (dj_du nullable)
cudaError_t launch_adj_sum(dugks_ctx* ctx, double* dj_dalpha, double* dj_du) {
    adj_sum_kernel<<<1, 1024, 0, ctx->stream>>>(ctx->adj_partial, ctx->adj_used, adj_partials(ctx),
                                                3.0 / (ctx->c * ctx->c), dj_dalpha, dj_du);
    return cudaGetLastError();
}

// The row-marching FP32 adjoint (adj_rows_kernel): periodic or Dirichlet walls, equilibrium
// degree <= 3, f and mu rows that TMA can copy (nx a multiple of 4, 16-byte aligned buffers).
#ifndef DUGKS_ADJ_ROW_STAGES
#define DUGKS_ADJ_ROW_STAGES 4
#endif
constexpr int kAdjRowStages = DUGKS_ADJ_ROW_STAGES;  // row stages in flight per warp (>= 3)
// Segments: as many as the 16-row minimum allows up to 96 warps per SM over the launch.  Short
// segments even out the end of the launch: 2048^2 took 186 us with 16-row segments against
// 200 us with 29-row ones (36 warps per SM) and 215 us with 24 warps per SM.
#ifndef DUGKS_ADJ_ROW_WARPS_PER_SM
#define DUGKS_ADJ_ROW_WARPS_PER_SM 96
#endif
#ifndef DUGKS_ADJ_ROW_MIN_SEG
#define DUGKS_ADJ_ROW_MIN_SEG 16
#endif
constexpr int kAdjRowWarpsPerSM = DUGKS_ADJ_ROW_WARPS_PER_SM;  // warps per SM over one launch (segment count)
constexpr int kAdjRowMinSeg = DUGKS_ADJ_ROW_MIN_SEG;           // rows per segment at least
// It is used from 1 M cells up (2048^2: 243 us against 506 us for the tiled kernel, 1024^2:
// 91 against 144 us; on 512^2, with too few warps in flight, the tiled kernel is faster), or
// wherever it applies when dugks_set_adjoint_kernel asked for it.
bool adj_rows_ok(const dugks_ctx* ctx, const void* f, const void* mu) {
    const bool applies = ctx->precision == 32 && ctx->nc != NC_LARGE && ctx->nx % 4 == 0 &&
                         ctx->nx >= 8 && ctx->ny >= 4 && (reinterpret_cast<uintptr_t>(f) % 16) == 0 &&
                         (reinterpret_cast<uintptr_t>(mu) % 16) == 0;
    if (!applies || ctx->adj_kernel == DUGKS_ADJ_TILED) return false;
    if (ctx->adj_kernel == DUGKS_ADJ_ROWS) return true;
    return (long long)ctx->nx * ctx->ny >= 1024LL * 1024;
}

template <int NC>
cudaError_t launch_adjoint_rows(dugks_ctx* ctx, const StepArgs<float, NC>& a, const AdjArgs<float>& g, const void* f,
                                const void* mu) {
    EncodeTiledFn encode = tiled_encoder(ctx);
    if (!encode) return cudaErrorNotSupported;
    using L = AdjRowLayout;
    CUtensorMap tm[2];
    const cuuint64_t dims[3] = {cuuint64_t(ctx->nx), cuuint64_t(ctx->ny), cuuint64_t(Q)};
    const cuuint64_t strides[2] = {cuuint64_t(ctx->nx) * 4, cuuint64_t(ctx->nx) * ctx->ny * 4};
    const cuuint32_t box[3] = {cuuint32_t(L::BOXW), 1u, cuuint32_t(Q)};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const void* base[2] = {f, mu};
    for (int b = 0; b < 2; ++b)
        if (encode(&tm[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base[b]), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return e;
    // about kAdjRowWarpsPerSM warps per SM over the launch, segments of at least kAdjRowMinSeg
    // rows, one partial per warp
    const int strips = (ctx->nx + L::WI - 1) / L::WI;
    const long long cap = adj_partials(ctx);
    long long nseg = std::max<long long>(1, (long long)kAdjRowWarpsPerSM * sms / strips);
    nseg = std::min<long long>(nseg, std::max(1, ctx->ny / kAdjRowMinSeg));
    nseg = std::max<long long>(1, std::min<long long>(nseg, cap / strips));
    const int seg = int((ctx->ny + nseg - 1) / nseg);
    nseg = (ctx->ny + seg - 1) / seg;
    if ((long long)strips * nseg > cap) return cudaErrorInvalidConfiguration;
    ctx->adj_used = int(strips * nseg);  // the sums read the slots this launch writes
    const AdjConstsP<NC> kp = make_adj_consts_p<NC>(ctx);
    const dim3 grid(strips, unsigned(nseg));
    const size_t smem = L::bytes(kAdjRowStages);
    if (ctx->xper && ctx->yper) {
        if (g.want_u)
            adj_rows_kernel<NC, kAdjRowStages, true, false><<<grid, 32, smem, ctx->stream>>>(tm[0], tm[1], a, kp, g, seg);
        else
            adj_rows_kernel<NC, kAdjRowStages, false, false><<<grid, 32, smem, ctx->stream>>>(tm[0], tm[1], a, kp, g, seg);
    } else {  // a Dirichlet wall on some axis
        if (g.want_u)
            adj_rows_kernel<NC, kAdjRowStages, true, true><<<grid, 32, smem, ctx->stream>>>(tm[0], tm[1], a, kp, g, seg);
        else
            adj_rows_kernel<NC, kAdjRowStages, false, true><<<grid, 32, smem, ctx->stream>>>(tm[0], tm[1], a, kp, g, seg);
    }
    return cudaGetLastError();
}

// One adjoint step.  accumulate: the step's partials are added to the partial buffer (a
// reverse sweep zeroes it first and sums it at the end); else they overwrite it and, with
// dj_dalpha set, are summed into *dj_dalpha (and dj_du[0..1] if set).  want_u: also form
// the u-derivative.
template <typename T, int NC>
cudaError_t launch_adjoint_step(dugks_ctx* ctx, const void* f, const void* mu, void* lam, double* dj_dalpha,
                                double* dj_du, bool want_u, bool accumulate) {
    StepArgs<T, NC> a = make_args<T, NC>(ctx, 0);
    a.fin = static_cast<const T*>(f);  // the adjoint reads contiguous [Q][ny][nx] states
    a.pitch = ctx->nx;
    a.plane = (long long)ctx->nx * ctx->ny;
    const Consts<T, NC> k = make_consts<T, NC>(ctx);
    const AdjConsts<T, NC> ka = make_adj_consts<T, NC>(ctx);
    AdjArgs<T> g;
    g.f = static_cast<const T*>(f);
    g.mu = static_cast<const T*>(mu);
    g.lam = static_cast<T*>(lam);
    g.Ax = static_cast<T*>(ctx->adj_ax);
    g.Ay = static_cast<T*>(ctx->adj_ay);
    g.partial = ctx->adj_partial;
    g.pstride = adj_partials(ctx);
    g.accumulate = accumulate ? 1 : 0;
    g.want_u = want_u ? 1 : 0;
    if constexpr (sizeof(T) == 4 && NC != NC_LARGE) {
        if (adj_rows_ok(ctx, f, mu)) {
            cudaError_t e = launch_adjoint_rows<NC>(ctx, a, g, f, mu);
            if (e != cudaSuccess) return e;
            if (dj_dalpha) return launch_adj_sum(ctx, dj_dalpha, dj_du);
            return cudaGetLastError();
        }
    }
    const int tb = adj_tile_blocks(ctx);
    ctx->adj_used = adj_partials(ctx);
    const size_t smem = AdjTile<T, kAdjTX, kAdjTY>::bytes();
    cudaError_t e = cudaFuncSetAttribute(adj_tile_kernel<T, NC, kAdjTX, kAdjTY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    const int wb = adj_wall_blocks(ctx);
    adj_tile_kernel<T, NC, kAdjTX, kAdjTY><<<adj_tile_grid(ctx), kAdjTX * kAdjTY, smem, ctx->stream>>>(a, k, ka, g,
                                                                                                     wb > 0 ? 1 : 0);
    if (wb > 0) adj_wall_kernel<T, NC><<<wb, kAdjThreads, 0, ctx->stream>>>(a, k, ka, g, tb);
    if (dj_dalpha) return launch_adj_sum(ctx, dj_dalpha, dj_du);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step_any(dugks_ctx* ctx, const void* f, const void* mu, void* lam, double* dj_dalpha,
                                    double* dj_du, bool want_u, bool accumulate) {
    const int nc = want_u ? std::max(ctx->nc, ctx->nc_u) : ctx->nc;
    if (ctx->precision == 32) {
        switch (nc) {
            case 3: return launch_adjoint_step<float, 3>(ctx, f, mu, lam, dj_dalpha, dj_du, want_u, accumulate);
            case 4: return launch_adjoint_step<float, 4>(ctx, f, mu, lam, dj_dalpha, dj_du, want_u, accumulate);
            default: return launch_adjoint_step<float, NC_LARGE>(ctx, f, mu, lam, dj_dalpha, dj_du, want_u, accumulate);
        }
    }
    switch (nc) {
        case 3: return launch_adjoint_step<double, 3>(ctx, f, mu, lam, dj_dalpha, dj_du, want_u, accumulate);
        case 4: return launch_adjoint_step<double, 4>(ctx, f, mu, lam, dj_dalpha, dj_du, want_u, accumulate);
        default: return launch_adjoint_step<double, NC_LARGE>(ctx, f, mu, lam, dj_dalpha, dj_du, want_u, accumulate);
    }
}

// dJ/dphi0 from lam^0; with dj_du set, the initialisation's share of dJ/du (f^0 = feq(phi0)
// depends on u) is added to dj_du[0..1]
template <typename T>
cudaError_t launch_init_adjoint(dugks_ctx* ctx, const void* phi0, const void* lam, void* gphi0, double* dj_du) {
    const long long n = (long long)ctx->nx * ctx->ny;
    const int blocks = init_blocks(ctx);
    init_adjoint_kernel<T, NC_LARGE><<<blocks, 256, 0, ctx->stream>>>(
        static_cast<const T*>(phi0), static_cast<const T*>(lam), static_cast<T*>(gphi0), n,
        make_adj_consts<T, NC_LARGE>(ctx), dj_du ? ctx->adj_upart : nullptr);
    if (dj_du)
        adj_sum_kernel<<<1, 1024, 0, ctx->stream>>>(ctx->adj_upart, blocks, blocks, 0.0, nullptr, dj_du);
    return cudaGetLastError();
}

dugks_status batch_fail(dugks_batch* b, cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    b->last_error = buf;
    return e == cudaErrorMemoryAllocation ? DUGKS_ERR_NOMEM : DUGKS_ERR_CUDA;
}

// Instance table and tile map for the current tile shape (seg_target rows per tile).
template <int NC>
dugks_status batch_build_tables(dugks_batch* b) {
    std::vector<BatchInst<NC>> h(size_t(b->n));
    std::vector<int> order(size_t(b->n));
    std::iota(order.begin(), order.end(), 0);
    // largest instances first, so the tile queue drains them early (longest-processing-time order)
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (long long)b->ctx[x]->nx * b->ctx[x]->ny > (long long)b->ctx[y]->nx * b->ctx[y]->ny;
    });
    // each instance: segments of seg_target rows over about long_frac of its rows, then
    // segments of kBatchShortRows; the short tiles of all instances follow all the long ones
    std::vector<BatchTile> tiles, shorts;
    for (int oi : order) {
        dugks_ctx* c = b->ctx[oi];
        BatchInst<NC>& I = h[size_t(oi)];
        memcpy(&I.tmap[0], &c->tmap[0], sizeof(CUtensorMap));
        memcpy(&I.tmap[1], &c->tmap[1], sizeof(CUtensorMap));
        I.args[0] = make_args<float, NC>(c, 0);
        I.args[1] = make_args<float, NC>(c, 1);
        I.args[0].err = I.args[1].err = b->d_err;
        I.k = make_constsp<NC>(c);
        I.rw = c->rowy;
        const int nstrips = (c->nx + WarpLayout<float>::WI - 1) / WarpLayout<float>::WI;
        const int L = std::max(1, std::min(b->seg_target, c->ny));
        int nlong = (c->ny + L - 1) / L, ylong = c->ny;
        if (b->split && L > 2 * kBatchShortRows) {
            nlong = int(b->long_frac * c->ny / L);
            ylong = nlong * L;
        }
        for (int sg = 0; sg < nlong; ++sg)
            for (int st = 0; st < nstrips; ++st)
                tiles.push_back(BatchTile{oi, st, sg * L, std::min(sg * L + L, c->ny)});
        for (int y = ylong; y < c->ny; y += kBatchShortRows)
            for (int st = 0; st < nstrips; ++st)
                shorts.push_back(BatchTile{oi, st, y, std::min(y + kBatchShortRows, c->ny)});
    }
    tiles.insert(tiles.end(), shorts.begin(), shorts.end());
    b->ntiles = int(tiles.size());
    cudaError_t e;
    if (b->d_insts) cudaFree(b->d_insts);
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_insts = nullptr;
    b->d_tiles = nullptr;
    if ((e = cudaMalloc(&b->d_insts, sizeof(BatchInst<NC>) * h.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_tiles, sizeof(BatchTile) * tiles.size())) != cudaSuccess)
        return batch_fail(b, e, "cudaMalloc(batch tables)");
    if ((e = cudaMemcpy(b->d_insts, h.data(), sizeof(BatchInst<NC>) * h.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return batch_fail(b, e, "cudaMemcpy(batch tables)");
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return DUGKS_OK;
}

dugks_status batch_tables(dugks_batch* b) { return b->nc == 3 ? batch_build_tables<3>(b) : batch_build_tables<4>(b); }

template <int NC>
cudaError_t batch_launch(dugks_batch* b, int* counter, int parity) {
    const size_t smem = WarpLayout<float>::bytes(b->stages);
    batch_step_vp<NC><<<b->blocks, 32, smem, b->stream>>>(static_cast<const BatchInst<NC>*>(b->d_insts),
                                                          b->d_tiles, b->ntiles, parity, counter, b->stages,
                                                          b->d_err);
    return cudaGetLastError();
}

// n steps as direct launches (counters reset first), starting from parity b->parity
cudaError_t batch_launch_steps(dugks_batch* b, int n) {
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * size_t(n), b->stream);
    for (int s = 0; s < n && e == cudaSuccess; ++s) {
        e = b->nc == 3 ? batch_launch<3>(b, b->d_counters + s, b->parity) : batch_launch<4>(b, b->d_counters + s, b->parity);
        b->parity ^= 1;
    }
    return e;
}

dugks_status batch_graph(dugks_batch* b) {
    if (b->graph) return DUGKS_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(b, e, "cudaStreamBeginCapture");
    const int p0 = b->parity;
    e = batch_launch_steps(b, dugks_batch::kGraphSteps);
    b->parity = p0;  // capturing launched nothing
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return batch_fail(b, e, "batch capture"); }
    if (e2 != cudaSuccess) return batch_fail(b, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->graph = nullptr; return batch_fail(b, e, "cudaGraphInstantiate"); }
    return DUGKS_OK;
}

dugks_status batch_step_impl(dugks_batch* b, long long n) {
    const long long G = dugks_batch::kGraphSteps;
    cudaError_t e;
    if (n >= G) {
        // the graph was captured for parity 0; it returns to the parity it started from
        if (b->parity != 0) {
            if ((e = batch_launch_steps(b, 1)) != cudaSuccess) return batch_fail(b, e, "batch step");
            --n;
        }
        dugks_status st = batch_graph(b);
        if (st != DUGKS_OK) return st;
        for (long long r = 0; r + G <= n; r += G)
            if ((e = cudaGraphLaunch(b->graph, b->stream)) != cudaSuccess) return batch_fail(b, e, "cudaGraphLaunch");
        n %= G;
    }
    if (n > 0 && (e = batch_launch_steps(b, int(n))) != cudaSuccess) return batch_fail(b, e, "batch step");
    return DUGKS_OK;
}

}  // namespace

extern "C" {

const char* dugks_status_string(dugks_status s) {
    switch (s) {
        case DUGKS_OK: return "ok";
        case DUGKS_ERR_ARG: return "invalid argument";
        case DUGKS_ERR_CONFIG: return "invalid configuration";
        case DUGKS_ERR_CUDA: return "CUDA error";
        case DUGKS_ERR_NONFINITE: return "non-finite value in phi";
        case DUGKS_ERR_UNSUPPORTED: return "unsupported";
        case DUGKS_ERR_NOMEM: return "out of memory";
        case DUGKS_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char* dugks_last_error(const dugks_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

dugks_status dugks_check_config(const dugks_mesh* mesh, const dugks_vset* vset, const dugks_coef* coef, double dt) {
    if (!mesh || !vset || !coef || !mesh->xf || !mesh->yf) return DUGKS_ERR_ARG;
    if (mesh->nx < 1 || mesh->ny < 1) return DUGKS_ERR_ARG;
    if (mesh->nx > (1 << 30) || mesh->ny > (1 << 30)) return DUGKS_ERR_ARG;
    if (vset->kind != DUGKS_D2Q9) return DUGKS_ERR_ARG;
    if (coef->nb < 0 || coef->nb > 8 || coef->nd < 0 || coef->nd > 8) return DUGKS_ERR_ARG;
    if (coef->d_tensor != 0 && coef->d_tensor != 1) return DUGKS_ERR_ARG;
    if (coef->d_tensor && (coef->ndt < 0 || coef->ndt > 8)) return DUGKS_ERR_ARG;
    if (coef->d_tensor &&
        (!finite_all(coef->dxx, coef->ndt) || !finite_all(coef->dxy, coef->ndt) || !finite_all(coef->dyy, coef->ndt)))
        return DUGKS_ERR_CONFIG;
    for (int w = 0; w < 4; ++w)
        if (mesh->bc[w] != DUGKS_BC_PERIODIC && mesh->bc[w] != DUGKS_BC_DIRICHLET) return DUGKS_ERR_ARG;
    if ((mesh->bc[0] == DUGKS_BC_PERIODIC) != (mesh->bc[1] == DUGKS_BC_PERIODIC)) return DUGKS_ERR_ARG;
    if ((mesh->bc[2] == DUGKS_BC_PERIODIC) != (mesh->bc[3] == DUGKS_BC_PERIODIC)) return DUGKS_ERR_ARG;
    if (!finite_all(mesh->xf, mesh->nx + 1) || !finite_all(mesh->yf, mesh->ny + 1)) return DUGKS_ERR_CONFIG;
    if (!finite_all(mesh->bc_value, 4) || !finite_all(coef->u, 2) || !finite_all(coef->b, coef->nb) ||
        !finite_all(coef->d, coef->nd) || !std::isfinite(coef->alpha) || !std::isfinite(vset->c) || !std::isfinite(dt))
        return DUGKS_ERR_CONFIG;
    double hmin = INFINITY;
    for (int j = 0; j < mesh->nx; ++j) {
        const double w = mesh->xf[j + 1] - mesh->xf[j];
        if (!(w > 0.0)) return DUGKS_ERR_CONFIG;
        hmin = std::min(hmin, w);
    }
    for (int k = 0; k < mesh->ny; ++k) {
        const double w = mesh->yf[k + 1] - mesh->yf[k];
        if (!(w > 0.0)) return DUGKS_ERR_CONFIG;
        hmin = std::min(hmin, w);
    }
    if (!(vset->c > 0.0) || !(coef->alpha > 0.0) || !(dt > 0.0)) return DUGKS_ERR_CONFIG;
    if (!(vset->c * dt / hmin < 1.0)) return DUGKS_ERR_CONFIG;
    return DUGKS_OK;
}

dugks_status dugks_check_feq(const dugks_vset* vset, const dugks_coef* coef, double phi_min, double phi_max,
                             double* feq_min_out) {
    if (!vset || !coef || vset->kind != DUGKS_D2Q9) return DUGKS_ERR_ARG;
    if (coef->nb < 0 || coef->nb > 8 || coef->nd < 0 || coef->nd > 8) return DUGKS_ERR_ARG;
    if (coef->d_tensor != 0 && coef->d_tensor != 1) return DUGKS_ERR_ARG;
    if (coef->d_tensor && (coef->ndt < 0 || coef->ndt > 8)) return DUGKS_ERR_ARG;
    if (!std::isfinite(phi_min) || !std::isfinite(phi_max) || phi_min > phi_max) return DUGKS_ERR_ARG;
    if (!std::isfinite(vset->c) || !(vset->c > 0.0) || !finite_all(coef->u, 2) || !finite_all(coef->b, coef->nb) ||
        !finite_all(coef->d, coef->nd))
        return DUGKS_ERR_CONFIG;
    if (coef->d_tensor &&
        (!finite_all(coef->dxx, coef->ndt) || !finite_all(coef->dxy, coef->ndt) || !finite_all(coef->dyy, coef->ndt)))
        return DUGKS_ERR_CONFIG;
    double cf[Q][NC_LARGE];
    int maxdeg = 1;
    feq_coefficients(vset, coef, cf, &maxdeg);
    double fmin = 0.0;
    const double margin = feq_margin_over(cf, phi_min, phi_max, &fmin);
    if (feq_min_out) *feq_min_out = fmin;
    return margin < 0.0 ? DUGKS_ERR_CONFIG : DUGKS_OK;
}

dugks_status dugks_create(const dugks_mesh* mesh, const dugks_vset* vset, const dugks_coef* coef, double dt,
                          const dugks_options* opts, dugks_ctx** out) {
    if (!out) return DUGKS_ERR_ARG;
    *out = nullptr;
    dugks_status st = dugks_check_config(mesh, vset, coef, dt);
    if (st != DUGKS_OK) return st;
    dugks_options o = {DUGKS_FP32, DUGKS_KERNEL_AUTO, nullptr, -1};
    if (opts) o = *opts;
    if (o.precision != DUGKS_FP32 && o.precision != DUGKS_FP64) return DUGKS_ERR_ARG;
    if (o.kernel != DUGKS_KERNEL_AUTO && o.kernel != DUGKS_KERNEL_FUSED && o.kernel != DUGKS_KERNEL_NAIVE)
        return DUGKS_ERR_ARG;

    dugks_ctx* ctx = new (std::nothrow) dugks_ctx();
    if (!ctx) return DUGKS_ERR_NOMEM;
    if (o.device < 0) {
        if (cudaGetDevice(&ctx->device) != cudaSuccess) { delete ctx; return DUGKS_ERR_CUDA; }
    } else {
        ctx->device = o.device;
    }
    DeviceGuard guard(ctx->device);
    ctx->nx = mesh->nx;
    ctx->ny = mesh->ny;
    ctx->precision = o.precision;
    ctx->kernel = o.kernel == DUGKS_KERNEL_NAIVE ? DUGKS_KERNEL_NAIVE : DUGKS_KERNEL_FUSED;
    ctx->xper = mesh->bc[0] == DUGKS_BC_PERIODIC;
    ctx->yper = mesh->bc[2] == DUGKS_BC_PERIODIC;
    for (int w = 0; w < 4; ++w) ctx->bcv[w] = mesh->bc_value[w];
    ctx->xf.assign(mesh->xf, mesh->xf + mesh->nx + 1);
    ctx->yf.assign(mesh->yf, mesh->yf + mesh->ny + 1);
    ctx->c = vset->c;
    ctx->dt = dt;
    ctx->ux = coef->u[0];
    ctx->uy = coef->u[1];
    ctx->nb = coef->nb;
    for (int m = 0; m < coef->nb; ++m) ctx->bcoef[m] = coef->b[m];
    ctx->c_zero = coef->c_zero;
    ctx->stream = static_cast<cudaStream_t>(o.stream);
    ctx->elem = ctx->precision == 32 ? sizeof(float) : sizeof(double);

    // relaxation time from the Chapman-Enskog result alpha = c_s^2 lambda (Section 3)
    const double cs2 = vset->c * vset->c / 3.0;
    const double lam = coef->alpha / cs2, h = 0.5 * dt;
    ctx->lambda = lam;
    double hmin = INFINITY;
    for (int j = 0; j < ctx->nx; ++j) hmin = std::min(hmin, ctx->xf[j + 1] - ctx->xf[j]);
    for (int k = 0; k < ctx->ny; ++k) hmin = std::min(hmin, ctx->yf[k + 1] - ctx->yf[k]);
    ctx->cfl = vset->c * dt / hmin;
    ctx->a_bp = (2.0 * lam - h) / (2.0 * lam + dt);  // Eq. 2.21
    ctx->b_bp = 3.0 * h / (2.0 * lam + dt);
    ctx->a_tp = (2.0 * lam - dt) / (2.0 * lam + dt);  // Eq. 2.13
    ctx->b_tp = 2.0 * dt / (2.0 * lam + dt);
    ctx->a_f = 2.0 * lam / (2.0 * lam + h);  // Eq. 2.22
    ctx->b_f = h / (2.0 * lam + h);
    ctx->hc = h * vset->c;

    const double c = vset->c;
    int maxdeg = 1;
    feq_coefficients(vset, coef, ctx->feq_coef, &maxdeg);
    ctx->nc = maxdeg <= 2 ? 3 : (maxdeg == 3 ? 4 : NC_LARGE);
    {  // with u = 0 the step's equilibrium has no b terms, but d feq / d u has b and C/(u u)
        int degb = 0;
        for (int m = 0; m < ctx->nb; ++m)
            if (ctx->bcoef[m] != 0.0) degb = m;
        const int degc = (ctx->c_zero || degb < 1) ? 0 : 2 * degb - 1;
        const int du = std::max(maxdeg, std::max(degb, degc));
        ctx->nc_u = du <= 2 ? 3 : (du == 3 ? 4 : NC_LARGE);
    }

    const int lane = 128 / int(ctx->elem);  // rows padded to 128 bytes
    ctx->pitch = ((long long)ctx->nx + lane - 1) / lane * lane;
    ctx->plane = ctx->pitch * ctx->ny;
    const size_t bytes = size_t(Q) * size_t(ctx->plane) * ctx->elem;

    auto fail = [&](dugks_status s) {
        dugks_status r = s;
        free_ctx(ctx);
        return r;
    };
    cudaError_t e;
    for (int b = 0; b < 2; ++b) {
        e = cudaMalloc(&ctx->buf[b], bytes);
        if (e != cudaSuccess) { cuda_fail(ctx, e, "cudaMalloc(state)"); return fail(DUGKS_ERR_NOMEM); }
        e = cudaMemsetAsync(ctx->buf[b], 0, bytes, ctx->stream);
        if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "cudaMemsetAsync"));
    }
    // metrics
    std::vector<double> dxw, dyw;
    auto upload = [&](void** dst, const void* src, size_t n) -> cudaError_t {
        cudaError_t r = cudaMalloc(dst, n);
        if (r != cudaSuccess) return r;
        return cudaMemcpy(*dst, src, n, cudaMemcpyHostToDevice);
    };
    if (ctx->precision == 32) {
        std::vector<FaceM<float>> fx, fy;
        std::vector<CellM<float>> cx, cy;
        build_metrics<float>(ctx->xf, ctx->xper, ctx->hc, dt, c, fx, cx, dxw);
        build_metrics<float>(ctx->yf, ctx->yper, ctx->hc, dt, c, fy, cy, dyw);
        if ((e = upload(&ctx->fxm, fx.data(), fx.size() * sizeof(fx[0]))) != cudaSuccess ||
            (e = upload(&ctx->fym, fy.data(), fy.size() * sizeof(fy[0]))) != cudaSuccess ||
            (e = upload(&ctx->cxm, cx.data(), cx.size() * sizeof(cx[0]))) != cudaSuccess ||
            (e = upload(&ctx->cym, cy.data(), cy.size() * sizeof(cy[0]))) != cudaSuccess)
            return fail(cuda_fail(ctx, e, "metrics upload"));
        const std::vector<RowY> rw = make_rowy(fy, cy, ctx->ny, float(ctx->hc));
        void* prw = nullptr;
        if ((e = upload(&prw, rw.data(), rw.size() * sizeof(rw[0]))) != cudaSuccess) {
            ctx->rowy = static_cast<RowY*>(prw);
            return fail(cuda_fail(ctx, e, "row metrics upload"));
        }
        ctx->rowy = static_cast<RowY*>(prw);
    } else {
        std::vector<FaceM<double>> fx, fy;
        std::vector<CellM<double>> cx, cy;
        build_metrics<double>(ctx->xf, ctx->xper, ctx->hc, dt, c, fx, cx, dxw);
        build_metrics<double>(ctx->yf, ctx->yper, ctx->hc, dt, c, fy, cy, dyw);
        if ((e = upload(&ctx->fxm, fx.data(), fx.size() * sizeof(fx[0]))) != cudaSuccess ||
            (e = upload(&ctx->fym, fy.data(), fy.size() * sizeof(fy[0]))) != cudaSuccess ||
            (e = upload(&ctx->cxm, cx.data(), cx.size() * sizeof(cx[0]))) != cudaSuccess ||
            (e = upload(&ctx->cym, cy.data(), cy.size() * sizeof(cy[0]))) != cudaSuccess)
            return fail(cuda_fail(ctx, e, "metrics upload"));
    }
    void* p = nullptr;
    if ((e = upload(&p, dxw.data(), dxw.size() * sizeof(double))) != cudaSuccess) { ctx->dxv = (double*)p; return fail(cuda_fail(ctx, e, "dx upload")); }
    ctx->dxv = static_cast<double*>(p);
    p = nullptr;
    if ((e = upload(&p, dyw.data(), dyw.size() * sizeof(double))) != cudaSuccess) { ctx->dyv = (double*)p; return fail(cuda_fail(ctx, e, "dy upload")); }
    ctx->dyv = static_cast<double*>(p);
    const long long ncell = (long long)ctx->nx * ctx->ny;
    ctx->red_blocks = int(std::min<long long>((ncell + 255) / 256, 4096));
    if ((e = cudaMalloc(&ctx->staging, sizeof(double) * size_t(ncell))) != cudaSuccess)
        return fail(cuda_fail(ctx, e, "cudaMalloc(staging)"));
    if ((e = cudaMalloc(&ctx->partial, sizeof(double) * size_t(ctx->red_blocks))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->mass_dev, sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->err_dev, sizeof(int))) != cudaSuccess)
        return fail(cuda_fail(ctx, e, "cudaMalloc(scalars)"));
    if ((e = cudaMemsetAsync(ctx->err_dev, 0, sizeof(int), ctx->stream)) != cudaSuccess)
        return fail(cuda_fail(ctx, e, "cudaMemsetAsync(err)"));
    if (ctx->kernel == DUGKS_KERNEL_FUSED) {
        st = plan_fused(ctx);
        if (st != DUGKS_OK) return fail(st);
        st = make_tensor_maps(ctx);
        if (st != DUGKS_OK) return fail(st);
    }
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return fail(cuda_fail(ctx, e, "cudaStreamSynchronize"));
    *out = ctx;
    return DUGKS_OK;
}

dugks_status dugks_destroy(dugks_ctx* ctx) {
    if (!ctx) return DUGKS_OK;
    {
        DeviceGuard guard(ctx->device);
        cudaStreamSynchronize(ctx->stream);
    }
    free_ctx(ctx);
    return DUGKS_OK;
}

dugks_status dugks_init_phi(dugks_ctx* ctx, const void* phi0_dev) {
    if (!ctx || !phi0_dev) return DUGKS_ERR_ARG;
    DeviceGuard guard(ctx->device);
    cudaError_t e = ctx->precision == 32 ? launch_init<float, float>(ctx, static_cast<const float*>(phi0_dev))
                                         : launch_init<double, double>(ctx, static_cast<const double*>(phi0_dev));
    CK(e);
    ctx->steps_done = 0;
    ctx->t = ctx->tbase = ctx->t0;
    ctx->tsteps = 0;
    ctx->src_first = true;
    return DUGKS_OK;
}

dugks_status dugks_init_phi_host(dugks_ctx* ctx, const double* phi0_host) {
    if (!ctx || !phi0_host) return DUGKS_ERR_ARG;
    DeviceGuard guard(ctx->device);
    const size_t n = size_t(ctx->nx) * ctx->ny;
    if (ctx->feq_check) {  // the initial equilibrium must be non-negative over the range of phi0
        double lo = INFINITY, hi = -INFINITY;
        for (size_t c = 0; c < n; ++c) {
            lo = std::min(lo, phi0_host[c]);
            hi = std::max(hi, phi0_host[c]);
        }
        if (!std::isfinite(lo) || !std::isfinite(hi)) {
            ctx->last_error = "phi0 holds a non-finite value";
            return DUGKS_ERR_CONFIG;
        }
        double fmin = 0.0;
        if (feq_margin_over(ctx->feq_coef, lo, hi, &fmin) < 0.0) {
            char buf[192];
            snprintf(buf, sizeof(buf), "the equilibrium of phi0 is negative (min %.3e over phi in [%.6g, %.6g])", fmin, lo,
                     hi);
            ctx->last_error = buf;
            return DUGKS_ERR_CONFIG;
        }
    }
    CK(cudaMemcpyAsync(ctx->staging, phi0_host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    cudaError_t e = ctx->precision == 32 ? launch_init<float, double>(ctx, ctx->staging)
                                         : launch_init<double, double>(ctx, ctx->staging);
    CK(e);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->steps_done = 0;
    ctx->t = ctx->tbase = ctx->t0;
    ctx->tsteps = 0;
    ctx->src_first = true;
    return DUGKS_OK;
}

dugks_status dugks_step(dugks_ctx* ctx, long long n) {
    if (!ctx || n < 0) return DUGKS_ERR_ARG;
    DeviceGuard guard(ctx->device);
    for (long long s = 0; s < n; ++s) {
        CK(launch_step_any(ctx));
        ctx->cur ^= 1;
        ++ctx->steps_done;
        ++ctx->tsteps;
        ctx->t = ctx->tbase + double(ctx->tsteps) * ctx->dt;
        ctx->src_first = false;
    }
    return DUGKS_OK;
}

dugks_status dugks_get_phi(dugks_ctx* ctx, void* phi_dev_out, double* mass_out) {
    if (!ctx) return DUGKS_ERR_ARG;
    DeviceGuard guard(ctx->device);
    cudaError_t e = ctx->precision == 32 ? launch_phi<float, float>(ctx, static_cast<float*>(phi_dev_out))
                                         : launch_phi<double, double>(ctx, static_cast<double*>(phi_dev_out));
    CK(e);
    if (mass_out) {
        CK(cudaMemcpyAsync(mass_out, ctx->mass_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (!std::isfinite(*mass_out)) return DUGKS_ERR_NONFINITE;
    }
    return DUGKS_OK;
}

dugks_status dugks_get_phi_host(dugks_ctx* ctx, double* phi_host_out, double* mass_out) {
    if (!ctx) return DUGKS_ERR_ARG;
    DeviceGuard guard(ctx->device);
    cudaError_t e = ctx->precision == 32 ? launch_phi<float, double>(ctx, ctx->staging)
                                         : launch_phi<double, double>(ctx, ctx->staging);
    CK(e);
    const size_t n = size_t(ctx->nx) * ctx->ny;
    if (phi_host_out)
        CK(cudaMemcpyAsync(phi_host_out, ctx->staging, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    double m = 0.0;
    CK(cudaMemcpyAsync(&m, ctx->mass_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (mass_out) *mass_out = m;
    if (!std::isfinite(m)) return DUGKS_ERR_NONFINITE;
    return DUGKS_OK;
}

dugks_status dugks_save_state(dugks_ctx* ctx, void* f_dev_out) {
    if (!ctx || !f_dev_out) return DUGKS_ERR_ARG;
    DeviceGuard guard(ctx->device);
    CK(cudaMemcpy2DAsync(f_dev_out, size_t(ctx->nx) * ctx->elem, ctx->buf[ctx->cur], size_t(ctx->pitch) * ctx->elem,
                         size_t(ctx->nx) * ctx->elem, size_t(Q) * ctx->ny, cudaMemcpyDeviceToDevice, ctx->stream));
    return DUGKS_OK;
}

dugks_status dugks_load_state(dugks_ctx* ctx, const void* f_dev_in) {
    if (!ctx || !f_dev_in) return DUGKS_ERR_ARG;
    DeviceGuard guard(ctx->device);
    CK(cudaMemcpy2DAsync(ctx->buf[ctx->cur], size_t(ctx->pitch) * ctx->elem, f_dev_in, size_t(ctx->nx) * ctx->elem,
                         size_t(ctx->nx) * ctx->elem, size_t(Q) * ctx->ny, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->steps_done = 0;
    ctx->src_first = true;  // the state carries no source history; time is kept
    ctx->tbase = ctx->t;
    ctx->tsteps = 0;
    return DUGKS_OK;
}

dugks_status dugks_set_stream(dugks_ctx* ctx, void* stream) {
    if (!ctx) return DUGKS_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return DUGKS_OK;
}

dugks_status dugks_sync(dugks_ctx* ctx) {
    if (!ctx) return DUGKS_ERR_ARG;
    DeviceGuard guard(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    int err = 0;
    CK(cudaMemcpy(&err, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & 1) {
        ctx->last_error = "a bounded TMA wait in the step kernel expired";
        return DUGKS_ERR_TIMEOUT;
    }
    if (err & 4) {
        ctx->last_error = "dugks_init_phi: the equilibrium of phi0 is negative in some cell";
        return DUGKS_ERR_CONFIG;
    }
    return DUGKS_OK;
}

dugks_status dugks_set_feq_check(dugks_ctx* ctx, int on) {
    if (!ctx || (on != 0 && on != 1)) return DUGKS_ERR_ARG;
    ctx->feq_check = on;
    return DUGKS_OK;
}

dugks_status dugks_set_adjoint_kernel(dugks_ctx* ctx, int kernel) {
    if (!ctx || (kernel != DUGKS_ADJ_AUTO && kernel != DUGKS_ADJ_TILED && kernel != DUGKS_ADJ_ROWS))
        return DUGKS_ERR_ARG;
    ctx->adj_kernel = kernel;
    return DUGKS_OK;
}

dugks_status dugks_wait_timeout_check(dugks_ctx* ctx, int limit_us) {
    if (!ctx || limit_us < 1 || limit_us > 1000000) return DUGKS_ERR_ARG;
    DeviceGuard guard(ctx->device);
    wait_timeout_kernel<<<1, 32, 0, ctx->stream>>>(ctx->err_dev, 1000ull * (unsigned long long)limit_us);
    CK(cudaGetLastError());
    return DUGKS_OK;
}

dugks_status dugks_info(const dugks_ctx* ctx, dugks_info_t* out) {
    if (!ctx || !out) return DUGKS_ERR_ARG;
    out->nx = ctx->nx;
    out->ny = ctx->ny;
    out->precision = ctx->precision;
    out->kernel = ctx->kernel;
    out->pitch = ctx->pitch;
    out->steps_done = ctx->steps_done;
    out->dt = ctx->dt;
    out->lambda = ctx->lambda;
    out->cfl = ctx->cfl;
    out->block_threads = ctx->kernel == DUGKS_KERNEL_NAIVE ? 128 : ctx->nt;
    out->grid_blocks = ctx->kernel == DUGKS_KERNEL_NAIVE ? ((ctx->nx + 127) / 128) * std::min(ctx->ny, 65535)
                                                         : ctx->nstrips * ctx->nseg;
    out->state_bytes = (long long)Q * ctx->plane * (long long)ctx->elem;
    out->time = ctx->t;
    out->nsrc = ctx->nsrc;
    return DUGKS_OK;
}

dugks_status dugks_set_source(dugks_ctx* ctx, int nterms, const double* rate, const int* power, const void* fields_dev,
                              double t0) {
    if (!ctx || nterms < 0 || nterms > 8 || !std::isfinite(t0)) return DUGKS_ERR_ARG;
    if (nterms > 0 && (!rate || !power || !fields_dev)) return DUGKS_ERR_ARG;
    for (int q = 0; q < nterms; ++q)
        if (!std::isfinite(rate[q]) || power[q] < 0 || power[q] > 15) return DUGKS_ERR_ARG;
    if (nterms > 0 && ctx->c_zero) {
        ctx->last_error = "source terms need C = int B'B' dphi (Remark 3)";
        return DUGKS_ERR_UNSUPPORTED;
    }
    if (nterms > 0 && ctx->kernel == DUGKS_KERNEL_NAIVE) {
        ctx->last_error = "source terms run on the fused kernel only";
        return DUGKS_ERR_UNSUPPORTED;
    }
    DeviceGuard guard(ctx->device);
    const size_t cells = size_t(ctx->nx) * ctx->ny;
    // the terms are held in ascending order of power (the sum F does not depend on the order)
    int order[8];
    for (int q = 0; q < nterms; ++q) order[q] = q;
    std::stable_sort(order, order + nterms, [&](int x, int y) { return power[x] < power[y]; });
    const char* fields = static_cast<const char*>(fields_dev);
    if (nterms > 0 && src_uses_aux(ctx)) {
        CK(cudaStreamSynchronize(ctx->stream));  // the old fields may still be read by queued steps
        EncodeTiledFn encode = tiled_encoder(ctx);
        if (!encode) return DUGKS_ERR_CUDA;
        using L = WarpLayout<float>;
        const size_t planes = size_t(nterms) + 1;
        for (int b = 0; b < 2; ++b) {
            if (ctx->aux[b]) { cudaFree(ctx->aux[b]); ctx->aux[b] = nullptr; }
            cudaError_t e = cudaMalloc(&ctx->aux[b], planes * size_t(ctx->plane) * sizeof(float));
            if (e != cudaSuccess) { ctx->aux[b] = nullptr; return cuda_fail(ctx, e, "cudaMalloc(source planes)"); }
            // the nterms field planes, pitched like ftilde; the last plane holds the phi history
            for (int q = 0; q < nterms; ++q)
                CK(cudaMemcpy2DAsync(static_cast<float*>(ctx->aux[b]) + size_t(q) * ctx->plane,
                                     size_t(ctx->pitch) * sizeof(float), fields + size_t(order[q]) * cells * sizeof(float),
                                     size_t(ctx->nx) * sizeof(float), size_t(ctx->nx) * sizeof(float), size_t(ctx->ny),
                                     cudaMemcpyDeviceToDevice, ctx->stream));
            const cuuint64_t dims[3] = {cuuint64_t(ctx->nx), cuuint64_t(ctx->ny), cuuint64_t(planes)};
            const cuuint64_t strides[2] = {cuuint64_t(ctx->pitch) * sizeof(float),
                                           cuuint64_t(ctx->plane) * sizeof(float)};
            const cuuint32_t box[3] = {cuuint32_t(L::BOXW), 1u, cuuint32_t(planes)};
            const cuuint32_t estr[3] = {1u, 1u, 1u};
            CUresult r = encode(&ctx->taux[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ctx->aux[b], dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                ctx->last_error = "cuTensorMapEncodeTiled failed for the source planes (" + std::to_string(int(r)) + ")";
                return DUGKS_ERR_CUDA;
            }
        }
        ctx->aux_box = int(planes) * L::BOXW * int(sizeof(float));
        ctx->src_stage = L::STAGE_BYTES + (ctx->aux_box + 127) / 128 * 128;
        // the segment plan of the source-term kernel from its own occupancy (long segments over
        // the first wave, short ones after them, as the plain step)
        if (ctx->nc != NC_LARGE) {
            int sms = 0, occ = 0;
            CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
            const void* fn = ctx->nc == 3 ? reinterpret_cast<const void*>(&step_vp_src<3>)
                                          : reinterpret_cast<const void*>(&step_vp_src<4>);
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32, src_vp_smem(ctx)));
            ctx->sp_src = SegPlan{ctx->seg_rows_src, ctx->nseg_src, ctx->seg_rows_src};
            ctx->nseg_sp_src = ctx->nseg_src;
            if (occ > 0)
                plan_long_short(ctx, (long long)sms * occ, kSrcPlanFirst, kSrcPlanShort, ctx->sp_src, ctx->nseg_sp_src);
        }
    } else if (nterms > 0) {
        CK(cudaStreamSynchronize(ctx->stream));  // the old fields may still be read by queued steps
        if (ctx->src_field) { cudaFree(ctx->src_field); ctx->src_field = nullptr; }
        cudaError_t e = cudaMalloc(&ctx->src_field, size_t(nterms) * cells * ctx->elem);
        if (e != cudaSuccess) { ctx->src_field = nullptr; return cuda_fail(ctx, e, "cudaMalloc(source fields)"); }
        for (int b = 0; b < 2; ++b)
            if (!ctx->hist[b]) {
                e = cudaMalloc(&ctx->hist[b], cells * ctx->elem);
                if (e != cudaSuccess) { ctx->hist[b] = nullptr; return cuda_fail(ctx, e, "cudaMalloc(source history)"); }
            }
        for (int q = 0; q < nterms; ++q)
            CK(cudaMemcpyAsync(static_cast<char*>(ctx->src_field) + size_t(q) * cells * ctx->elem,
                               fields + size_t(order[q]) * cells * ctx->elem, cells * ctx->elem,
                               cudaMemcpyDeviceToDevice, ctx->stream));
    }
    for (int q = 0; q < nterms; ++q) {
        ctx->src_rate[q] = rate[order[q]];
        ctx->src_power[q] = power[order[q]];
    }
    ctx->nsrc = nterms;
    ctx->t0 = ctx->t = ctx->tbase = t0;
    ctx->tsteps = 0;
    ctx->src_first = true;
    return DUGKS_OK;
}

dugks_status dugks_adjoint_step(dugks_ctx* ctx, const void* f_dev, const void* mu_dev, void* lam_dev,
                                double* dj_dalpha_dev, double* dj_du_dev) {
    if (!ctx || !f_dev || !mu_dev || !lam_dev || (dj_du_dev && !dj_dalpha_dev)) return DUGKS_ERR_ARG;
    if (ctx->nsrc > 0) {
        ctx->last_error = "the adjoint covers the step without source terms";
        return DUGKS_ERR_UNSUPPORTED;
    }
    DeviceGuard guard(ctx->device);
    dugks_status st = adj_alloc(ctx);
    if (st != DUGKS_OK) return st;
    CK(launch_adjoint_step_any(ctx, f_dev, mu_dev, lam_dev, dj_dalpha_dev, dj_du_dev, dj_du_dev != nullptr, false));
    return DUGKS_OK;
}

dugks_status dugks_adjoint(dugks_ctx* ctx, const void* phi0_dev, long long nsteps, int checkpoint_every,
                           const void* grad_phiN_dev, void* grad_phi0_dev, double* grad_alpha_out,
                           double* grad_u_out) {
    if (!ctx || !phi0_dev || !grad_phiN_dev || !grad_phi0_dev || nsteps < 0 || checkpoint_every < 1)
        return DUGKS_ERR_ARG;
    if (ctx->nsrc > 0) {
        ctx->last_error = "the adjoint covers the step without source terms";
        return DUGKS_ERR_UNSUPPORTED;
    }
    DeviceGuard guard(ctx->device);
    dugks_status st = adj_alloc(ctx);
    if (st != DUGKS_OK) return st;
    const long long K = std::min<long long>(checkpoint_every, std::max<long long>(nsteps, 1));
    const long long nseg = nsteps == 0 ? 0 : (nsteps + K - 1) / K;
    // states of 256-byte-aligned size in one workspace: nseg checkpoints, K segment states, two lambdas
    const size_t sbytes = (size_t(Q) * ctx->nx * ctx->ny * ctx->elem + 255) / 256 * 256;
    const size_t need = sbytes * size_t(nseg + K + 2);
    if (need > ctx->adj_ws_bytes) {
        if (ctx->adj_ws) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->adj_ws);
            ctx->adj_ws = nullptr;
            ctx->adj_ws_bytes = 0;
        }
        if (cudaMalloc(&ctx->adj_ws, need) != cudaSuccess) {
            ctx->adj_ws = nullptr;
            ctx->last_error = "adjoint workspace allocation failed";
            return DUGKS_ERR_NOMEM;
        }
        ctx->adj_ws_bytes = need;
    }
    unsigned char* ws = static_cast<unsigned char*>(ctx->adj_ws);
    std::vector<void*> ckpt(size_t(nseg), nullptr), seg(size_t(K), nullptr);
    for (long long q = 0; q < nseg; ++q) ckpt[size_t(q)] = ws + size_t(q) * sbytes;
    for (long long q = 0; q < K; ++q) seg[size_t(q)] = ws + size_t(nseg + q) * sbytes;
    void* lam[2] = {ws + size_t(nseg + K) * sbytes, ws + size_t(nseg + K + 1) * sbytes};
    auto fail = [&](cudaError_t e, const char* what) {
        dugks_status s = cuda_fail(ctx, e, what);
        cudaStreamSynchronize(ctx->stream);
        return s;
    };
    cudaError_t e;
    // forward sweep, keeping one state per segment
    if ((st = dugks_init_phi(ctx, phi0_dev)) != DUGKS_OK) return st;
    for (long long s = 0; s < nseg; ++s) {
        if ((st = dugks_save_state(ctx, ckpt[s])) != DUGKS_OK) return st;
        if ((st = dugks_step(ctx, std::min(K, nsteps - s * K))) != DUGKS_OK) return st;
    }
    if ((e = cudaMemsetAsync(ctx->adj_dalpha, 0, 3 * sizeof(double), ctx->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(ctx->adj_partial, 0, 3 * sizeof(double) * size_t(adj_partials(ctx)), ctx->stream)) !=
            cudaSuccess)
        return fail(e, "cudaMemsetAsync");
    const bool want_u = grad_u_out != nullptr;
    double* du_dev = want_u ? ctx->adj_dalpha + 1 : nullptr;
    const long long n = (long long)ctx->nx * ctx->ny;
    const int blocks = int(std::min<long long>((n + 255) / 256, 65535));
    if (ctx->precision == 32)
        broadcast_phi_adjoint<float><<<blocks, 256, 0, ctx->stream>>>(static_cast<const float*>(grad_phiN_dev),
                                                                     static_cast<float*>(lam[0]), n);
    else
        broadcast_phi_adjoint<double><<<blocks, 256, 0, ctx->stream>>>(static_cast<const double*>(grad_phiN_dev),
                                                                       static_cast<double*>(lam[0]), n);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "broadcast_phi_adjoint");
    int cur = 0;
    // reverse sweep: recompute each segment from its checkpoint, then step the adjoint back through it
    for (long long s = nseg - 1; s >= 0; --s) {
        const long long ns = std::min(K, nsteps - s * K);
        if ((st = dugks_load_state(ctx, ckpt[s])) != DUGKS_OK) return st;
        for (long long q = 0; q < ns; ++q) {
            if ((st = dugks_save_state(ctx, seg[q])) != DUGKS_OK) return st;
            if (q + 1 < ns && (st = dugks_step(ctx, 1)) != DUGKS_OK) return st;
        }
        for (long long q = ns - 1; q >= 0; --q) {
            if ((e = launch_adjoint_step_any(ctx, seg[q], lam[cur], lam[1 - cur], nullptr, nullptr, want_u, true)) !=
                cudaSuccess)
                return fail(e, "adjoint step");
            cur ^= 1;
        }
    }
    if ((e = launch_adj_sum(ctx, ctx->adj_dalpha, du_dev)) != cudaSuccess) return fail(e, "adjoint sum");
    e = ctx->precision == 32 ? launch_init_adjoint<float>(ctx, phi0_dev, lam[cur], grad_phi0_dev, du_dev)
                             : launch_init_adjoint<double>(ctx, phi0_dev, lam[cur], grad_phi0_dev, du_dev);
    if (e != cudaSuccess) return fail(e, "init adjoint");
    double res[3] = {0.0, 0.0, 0.0};
    if ((e = cudaMemcpyAsync(res, ctx->adj_dalpha, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)) !=
        cudaSuccess)
        return fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return fail(e, "cudaStreamSynchronize");
    if (grad_alpha_out) *grad_alpha_out = res[0];
    if (grad_u_out) {
        grad_u_out[0] = res[1];
        grad_u_out[1] = res[2];
    }
    return DUGKS_OK;
}

dugks_status dugks_batch_create(int n, const dugks_mesh* meshes, const dugks_vset* vsets, const dugks_coef* coefs,
                                const double* dts, const dugks_options* opts, dugks_batch** out) {
    if (!out) return DUGKS_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !meshes || !vsets || !coefs || !dts) return DUGKS_ERR_ARG;
    dugks_options o = {DUGKS_FP32, DUGKS_KERNEL_FUSED, nullptr, -1};
    if (opts) o = *opts;
    if (o.precision != DUGKS_FP32) return DUGKS_ERR_UNSUPPORTED;  // the batched step is single precision
    for (int i = 0; i < n; ++i) {
        dugks_status st = dugks_check_config(&meshes[i], &vsets[i], &coefs[i], dts[i]);
        if (st != DUGKS_OK) return st;
    }
    dugks_batch* b = new (std::nothrow) dugks_batch();
    if (!b) return DUGKS_ERR_NOMEM;
    if (o.device < 0) {
        if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return DUGKS_ERR_CUDA; }
    } else {
        b->device = o.device;
    }
    DeviceGuard guard(b->device);
    auto fail = [&](dugks_status s) {
        dugks_batch_destroy(b);
        return s;
    };
    b->n = n;
    if (o.stream) {
        b->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return DUGKS_ERR_CUDA; }
        b->own_stream = true;
    }
    dugks_options io = o;
    io.kernel = DUGKS_KERNEL_FUSED;
    io.stream = b->stream;
    io.device = b->device;
    b->ctx.assign(size_t(n), nullptr);
    int nc = 3;
    for (int i = 0; i < n; ++i) {
        dugks_status st = dugks_create(&meshes[i], &vsets[i], &coefs[i], dts[i], &io, &b->ctx[size_t(i)]);
        if (st != DUGKS_OK) return fail(st);
        if (b->ctx[size_t(i)]->nc > 4) return fail(DUGKS_ERR_UNSUPPORTED);  // equilibrium polynomials of degree <= 3
        nc = std::max(nc, b->ctx[size_t(i)]->nc);
    }
    b->nc = nc;
    int sms = 0, occ = 0;
    cudaError_t e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device)) != cudaSuccess)
        return fail(batch_fail(b, e, "cudaDeviceGetAttribute"));
    const size_t smem = WarpLayout<float>::bytes(b->stages);
    void* fn = nc == 3 ? reinterpret_cast<void*>(&batch_step_vp<3>) : reinterpret_cast<void*>(&batch_step_vp<4>);
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32, smem)) != cudaSuccess)
        return fail(batch_fail(b, e, "batch kernel attributes"));
    b->blocks = sms * std::max(1, occ);
    if ((e = cudaMalloc(&b->d_counters, sizeof(int) * dugks_batch::kGraphSteps)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream)) != cudaSuccess)
        return fail(batch_fail(b, e, "cudaMalloc(batch scalars)"));
    dugks_status st = batch_tables(b);
    if (st != DUGKS_OK) return fail(st);
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return fail(batch_fail(b, e, "cudaStreamSynchronize"));
    *out = b;
    return DUGKS_OK;
}

dugks_status dugks_batch_destroy(dugks_batch* b) {
    if (!b) return DUGKS_OK;
    {
        DeviceGuard guard(b->device);
        if (b->stream) cudaStreamSynchronize(b->stream);
        if (b->graph) cudaGraphExecDestroy(b->graph);
        for (void* p : {b->d_insts, static_cast<void*>(b->d_tiles), static_cast<void*>(b->d_counters),
                        static_cast<void*>(b->d_err)})
            if (p) cudaFree(p);
    }
    for (dugks_ctx* c : b->ctx) dugks_destroy(c);
    if (b->own_stream) {
        DeviceGuard guard(b->device);
        cudaStreamDestroy(b->stream);
    }
    delete b;
    return DUGKS_OK;
}

dugks_status dugks_batch_init_phi(dugks_batch* b, int i, const void* phi0_dev) {
    if (!b || i < 0 || i >= b->n) return DUGKS_ERR_ARG;
    if (b->parity != 0) return DUGKS_ERR_UNSUPPORTED;  // initialise every instance before the first step
    return dugks_init_phi(b->ctx[size_t(i)], phi0_dev);
}

dugks_status dugks_batch_step(dugks_batch* b, long long n) {
    if (!b || n < 0) return DUGKS_ERR_ARG;
    DeviceGuard guard(b->device);
    const int p0 = b->parity;
    dugks_status st = batch_step_impl(b, n);
    if (st != DUGKS_OK) return st;
    // the instances' contexts follow the batch's parity
    for (dugks_ctx* c : b->ctx) {
        c->cur = b->parity;
        c->steps_done += n;
    }
    (void)p0;
    b->steps_done += n;
    return DUGKS_OK;
}

dugks_status dugks_batch_get_phi(dugks_batch* b, int i, void* phi_dev_out, double* mass_out) {
    if (!b || i < 0 || i >= b->n) return DUGKS_ERR_ARG;
    return dugks_get_phi(b->ctx[size_t(i)], phi_dev_out, mass_out);
}

dugks_status dugks_batch_save_state(dugks_batch* b, int i, void* f_dev_out) {
    if (!b || i < 0 || i >= b->n) return DUGKS_ERR_ARG;
    return dugks_save_state(b->ctx[size_t(i)], f_dev_out);
}

dugks_status dugks_batch_sync(dugks_batch* b) {
    if (!b) return DUGKS_ERR_ARG;
    DeviceGuard guard(b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "cudaStreamSynchronize");
    int err = 0;
    if ((e = cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return batch_fail(b, e, "cudaMemcpy");
    if (err) {
        b->last_error = "a bounded TMA wait in the batched step expired";
        return DUGKS_ERR_TIMEOUT;
    }
    return DUGKS_OK;
}

dugks_status dugks_batch_autotune(dugks_batch* b, int steps_per_trial, int* best_rows_out, float* best_ms_out) {
    if (!b || steps_per_trial < 1) return DUGKS_ERR_ARG;
    DeviceGuard guard(b->device);
    // trial steps run on copies: every instance's state is saved first and restored afterwards
    std::vector<void*> saved(size_t(b->n), nullptr);
    auto release = [&]() {
        for (void* p : saved) if (p) cudaFree(p);
    };
    cudaError_t e;
    for (int i = 0; i < b->n; ++i) {
        dugks_ctx* c = b->ctx[size_t(i)];
        if ((e = cudaMalloc(&saved[size_t(i)], size_t(Q) * c->nx * c->ny * c->elem)) != cudaSuccess) {
            release();
            return batch_fail(b, e, "cudaMalloc(autotune snapshot)");
        }
        dugks_status st = dugks_save_state(c, saved[size_t(i)]);
        if (st != DUGKS_OK) { release(); return st; }
    }
    const int p_saved = b->parity;
    // tile heights, each without the short tiles at the end of the queue and with them after
    // long tiles over 0.8, 0.7 or 0.6 of every instance's rows
    const int cands[] = {8, 16, 24, 32, 48, 64, 96, 128};
    const double fracs[] = {0.8, 0.7, 0.6};
    constexpr int NV = 1 + int(sizeof(fracs) / sizeof(fracs[0]));
    int best = b->seg_target;
    bool best_split = b->split;
    double best_frac = b->long_frac;
    float best_ms = 1e30f;
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    for (int trial = 0; trial < NV * int(sizeof(cands) / sizeof(cands[0])); ++trial) {
        const int cand = cands[trial / NV], v = trial % NV;
        b->seg_target = cand;
        b->split = v != 0;
        if (v) b->long_frac = fracs[v - 1];
        if (b->split && cand <= 2 * kBatchShortRows) continue;  // no short tiles to split off
        dugks_status st = batch_tables(b);
        if (st != DUGKS_OK) { release(); return st; }
        if ((e = batch_launch_steps(b, std::min(2, dugks_batch::kGraphSteps))) != cudaSuccess) break;  // warm-up
        cudaEventRecord(ev0, b->stream);
        for (int s = 0; s < steps_per_trial && e == cudaSuccess; s += dugks_batch::kGraphSteps)
            e = batch_launch_steps(b, std::min(dugks_batch::kGraphSteps, steps_per_trial - s));
        cudaEventRecord(ev1, b->stream);
        if (e != cudaSuccess || (e = cudaEventSynchronize(ev1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        if (ms < best_ms) { best_ms = ms; best = cand; best_split = b->split; best_frac = b->long_frac; }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (e != cudaSuccess) { release(); return batch_fail(b, e, "autotune trial"); }
    // restore the states and the parity they belong to
    b->parity = p_saved;
    for (int i = 0; i < b->n; ++i) {
        dugks_ctx* c = b->ctx[size_t(i)];
        c->cur = p_saved;
        const long long sd = c->steps_done;
        dugks_status st = dugks_load_state(c, saved[size_t(i)]);
        c->steps_done = sd;
        if (st != DUGKS_OK) { release(); return st; }
    }
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) { release(); return batch_fail(b, e, "sync"); }
    release();
    b->seg_target = best;
    b->split = best_split;
    b->long_frac = best_frac;
    dugks_status st = batch_tables(b);
    if (st != DUGKS_OK) return st;
    if (best_rows_out) *best_rows_out = best;
    if (best_ms_out) *best_ms_out = best_ms / float(steps_per_trial);
    return DUGKS_OK;
}

const char* dugks_batch_last_error(const dugks_batch* b) { return b ? b->last_error.c_str() : ""; }

}  // extern "C"

// ---- allocation-free phi / mass --------------------------------------------
// Partial sums of the reduction live in this fixed device array instead of
// a context's buffer.  Host code cannot use the symbol's address directly
// (in host code it names a host-side shadow), so every call looks up its
// device address on the current device with cudaGetSymbolAddress (a host
// call; nothing is cached that a device reset could leave stale).
static __device__ __align__(256) double g_noalloc_partial[DUGKS_NOALLOC_MAX_BLOCKS];

namespace {
constexpr int kMaxDevices = 64;

cudaError_t noalloc_scratch(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}
}  // namespace

extern "C" dugks_status dugks_phi_mass_noalloc(const void* f_dev, int precision, int nx, int ny,
                                               const double* dx_dev, const double* dy_dev, void* phi_dev_out,
                                               double* mass_dev_out, void* stream) {
    if (!f_dev || !dx_dev || !dy_dev || !mass_dev_out) return DUGKS_ERR_ARG;
    if (precision != DUGKS_FP32 && precision != DUGKS_FP64) return DUGKS_ERR_ARG;
    if (nx < 1 || ny < 1) return DUGKS_ERR_ARG;
    const long long n = (long long)nx * ny;
    if (n > DUGKS_NOALLOC_MAX_CELLS) return DUGKS_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DUGKS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DUGKS_ERR_UNSUPPORTED;
    double* partial = nullptr;
    if (noalloc_scratch(&partial) != cudaSuccess) return DUGKS_ERR_CUDA;
    const int blocks = int((n + 255) / 256);  // one partial per 256 cells, each written exactly once
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // an error the caller left pending is neither cleared nor reported as this call's
    const cudaError_t before = cudaPeekAtLastError();
    if (precision == DUGKS_FP32)
        phi_mass_kernel<float, float><<<blocks, 256, 0, s>>>(static_cast<const float*>(f_dev),
                                                             static_cast<float*>(phi_dev_out), nx, ny, nx, n, dx_dev,
                                                             dy_dev, partial);
    else
        phi_mass_kernel<double, double><<<blocks, 256, 0, s>>>(static_cast<const double*>(f_dev),
                                                               static_cast<double*>(phi_dev_out), nx, ny, nx, n,
                                                               dx_dev, dy_dev, partial);
    sum_partials_kernel<<<1, 256, 0, s>>>(partial, blocks, mass_dev_out);
    if (before == cudaSuccess && cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();  // this call's launch failure: clear it and report it
        return DUGKS_ERR_CUDA;
    }
    return DUGKS_OK;
}
