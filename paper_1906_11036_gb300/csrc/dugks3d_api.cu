// dugks3d_api.cu -- host side of the 3-D C ABI (include/dugks3d.h): context,
// metrics, equilibrium polynomials of Eq. 2.3 per velocity, and launches of the
// kernels in dugks3d_kernels.cuh.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dugks3d.h"
#include "dugks3d_halves.cuh"

using namespace dugks3;

namespace {
constexpr int NCL = 16;  // coefficient capacity of the equilibrium polynomials
}

struct dugks_3d_ctx {
    int device = 0;
    int nx = 0, ny = 0, nz = 0, q = 19, precision = 32, nc = 4;
    int per[3] = {1, 1, 1};
    double bcv[6] = {0, 0, 0, 0, 0, 0};
    double c = 1, dt = 0, lambda = 0, cfl = 0;
    double feq_coef[19][NCL];
    double a_bp = 0, b_bp = 0, a_f = 0, b_f = 0, hc = 0;
    size_t elem = 4;
    cudaStream_t stream = nullptr;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    void* fm[3] = {nullptr, nullptr, nullptr};  // FaceM<T>[n+3] per axis
    void* cm[3] = {nullptr, nullptr, nullptr};  // CellM<T>[n+2] per axis
    double* width[3] = {nullptr, nullptr, nullptr};
    double* partial = nullptr;
    double* mass_dev = nullptr;
    int* err_dev = nullptr;  // device error word of the step kernel (bit 0: a bounded TMA wait expired)
    bool tma = false;        // FP32 with nx a multiple of 4: ftilde staged by TMA (tmap[b] maps buf[b])
    CUtensorMap tmap[2];
    int red_blocks = 0;
    int nw = 16, zseg = 1, grid[3] = {1, 1, 1};
    long long steps_done = 0;
    std::string last_error;
};

namespace {

struct Guard3 {
    int prev = -1;
    explicit Guard3(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard3() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

dugks_status fail3(dugks_3d_ctx* ctx, cudaError_t e, const char* what) {
    if (ctx) {
        char b[256];
        snprintf(b, sizeof(b), "%s: %s", what, cudaGetErrorString(e));
        ctx->last_error = b;
    }
    return e == cudaErrorMemoryAllocation ? DUGKS_ERR_NOMEM : DUGKS_ERR_CUDA;
}

#define CK3(call)                                                 \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return fail3(ctx, e_, #call);      \
    } while (0)

bool finite_n(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// D3Q15 (Eq. 2.28) and D3Q19 (Eq. 2.6) weights
double weight3(int q, int i) {
    if (q == 19) return i == 0 ? 1.0 / 3 : (i <= 6 ? 1.0 / 18 : 1.0 / 36);
    return i == 0 ? 2.0 / 9 : (i <= 6 ? 1.0 / 9 : 1.0 / 72);
}
int dir3(int q, int i, int a) { return q == 19 ? E3<19>(i, a) : E3<15>(i, a); }

// Face and cell metrics along one axis (faces f, periodic flag): see FaceM / CellM.
template <typename T>
void metrics3(const std::vector<double>& f, bool per, double hcv, double dt, double c, std::vector<FaceM<T>>& fm,
              std::vector<CellM<T>>& cm, std::vector<double>& width) {
    const int n = int(f.size()) - 1;
    std::vector<double> xc(n + 2);  // centres j = -1..n at index j+1
    for (int j = 0; j < n; ++j) xc[j + 1] = 0.5 * (f[j] + f[j + 1]);
    const double L = f[n] - f[0];
    if (per) {
        xc[0] = xc[n] - L;
        xc[n + 1] = xc[1] + L;
    } else {
        xc[0] = 2.0 * f[0] - xc[1];
        xc[n + 1] = 2.0 * f[n] - xc[n];
    }
    fm.assign(n + 3, FaceM<T>{T(0.5), T(0), T(0), T(0)});
    for (int q = 0; q <= n; ++q) {
        const double xl = xc[q], xr = xc[q + 1], dxc = xr - xl, w = (f[q] - xl) / dxc;
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

// (a, 1 - a) with a + b == 1 exactly in T (a in (-1, 1)): rounded weights keep the discrete mass
template <typename T>
void unit_pair3(double a_exact, T& a, T& b) {
    b = T(1.0 - double(T(a_exact)));
    a = T(1.0 - double(b));
}

template <typename T, int QQ, int NC>
Consts3<T, QQ, NC> consts3(const dugks_3d_ctx* ctx) {
    Consts3<T, QQ, NC> k;
    unit_pair3<T>(ctx->a_bp, k.a_bp, k.b_bp);
    for (int i = 0; i < QQ; ++i)
        for (int m = 0; m < NC; ++m) {
            k.feq[i][m] = T(ctx->feq_coef[i][m]);
            k.hbp[i][m] = T(double(k.b_bp) * ctx->feq_coef[i][m]);
            k.hf[i][m] = T(ctx->b_f * ctx->feq_coef[i][m]);
        }
    k.a_f = T(ctx->a_f);
    k.third = T(1.0 / 3.0);
    k.hc = T(ctx->hc);
    for (int w = 0; w < 6; ++w) k.bcv[w] = T(ctx->bcv[w]);
    return k;
}

// the pair constants of step3d_vp (FP32)
template <int QQ, int NC>
Consts3P<QQ, NC> consts3p(const dugks_3d_ctx* ctx) {
    const Consts3<float, QQ, NC> s = consts3<float, QQ, NC>(ctx);
    Consts3P<QQ, NC> k;
    for (int q = 0; q < Consts3P<QQ, NC>::NP; ++q)
        for (int m = 0; m < NC; ++m) {
            k.hbp[q][m] = make_float2(s.hbp[PA3<QQ>(q)][m], s.hbp[PB3<QQ>(q)][m]);
            k.hf[q][m] = make_float2(s.hf[PA3<QQ>(q)][m], s.hf[PB3<QQ>(q)][m]);
        }
    for (int i = 0; i < QQ; ++i)
        for (int m = 0; m < NC; ++m) k.feq[i][m] = s.feq[i][m];
    k.a_bp = s.a_bp;
    k.b_bp = s.b_bp;
    k.third = s.third;
    k.hc = s.hc;
    k.a_bp2 = make_float2(s.a_bp, s.a_bp);
    k.a_f2 = make_float2(s.a_f, s.a_f);
    k.third2 = make_float2(s.third, s.third);
    for (int w = 0; w < 6; ++w) k.bcv[w] = s.bcv[w];
    return k;
}

template <typename T>
Args3<T> args3(const dugks_3d_ctx* ctx) {
    Args3<T> a;
    a.fin = static_cast<const T*>(ctx->buf[ctx->cur]);
    a.fout = static_cast<T*>(ctx->buf[ctx->cur ^ 1]);
    a.nx = ctx->nx;
    a.ny = ctx->ny;
    a.nz = ctx->nz;
    a.plane = (long long)ctx->nx * ctx->ny * ctx->nz;
    for (int d = 0; d < 3; ++d) {
        a.per[d] = ctx->per[d];
        a.fm[d] = static_cast<const FaceM<T>*>(ctx->fm[d]);
        a.cm[d] = static_cast<const CellM<T>*>(ctx->cm[d]);
    }
    a.zseg = ctx->zseg;
    a.err = ctx->err_dev;
    return a;
}

typedef CUresult (*EncodeTiled3Fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 4-D maps (x, y, z, velocity) of the two FP32 state buffers, box 36 x 1 x 1 x Q (the TMA
// staging of step3d_vp); false where the driver entry point or the encoding is not available
bool encode_tmaps3(dugks_3d_ctx* ctx) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    auto encode = reinterpret_cast<EncodeTiled3Fn>(fn);
    const cuuint64_t dims[4] = {cuuint64_t(ctx->nx), cuuint64_t(ctx->ny), cuuint64_t(ctx->nz), cuuint64_t(ctx->q)};
    const cuuint64_t strides[3] = {cuuint64_t(ctx->nx) * 4, cuuint64_t(ctx->nx) * ctx->ny * 4,
                                   cuuint64_t(ctx->nx) * ctx->ny * ctx->nz * 4};
    const cuuint32_t box[4] = {cuuint32_t(BOX3W), 1u, 1u, cuuint32_t(ctx->q)};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    for (int b = 0; b < 2; ++b)
        if (encode(&ctx->tmap[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ctx->buf[b], dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    return true;
}

template <typename T, int QQ, int NC, int NW>
constexpr size_t smem3() {
    return size_t(3 * NW * QQ * 32 + NW * NCROSS * 32 + 3 * NW * 4 * 32 + 3 * NW * QQ * 32) * sizeof(T);
}

// FP32 runs the velocity-pair kernel, FP64 the scalar one
template <typename T, int QQ, int NC, int NW>
cudaError_t launch3(dugks_3d_ctx* ctx) {
    const dim3 grid(ctx->grid[0], ctx->grid[1], ctx->grid[2]);
    if constexpr (std::is_same<T, float>::value) {
        if (ctx->tma) {
            if constexpr (QQ == 15)  // the face-halves kernel (D3Q15 256^3: 1166 us against 1214)
                step3d_hv<QQ, NC, NW><<<grid, NW * 32, smem3_hv<QQ, NW>(), ctx->stream>>>(
                    ctx->tmap[ctx->cur], args3<float>(ctx), consts3p<QQ, NC>(ctx));
            else  // D3Q19: the face kernel on TMA boxes (256^3: 1132 us; the face-halves kernel 1188-1211)
                step3d_vp<QQ, NC, NW, true><<<grid, NW * 32, smem3_vp<QQ, NW, true>(), ctx->stream>>>(
                    ctx->tmap[ctx->cur], args3<float>(ctx), consts3p<QQ, NC>(ctx));
        }
        else
            step3d_vp<QQ, NC, NW, false><<<grid, NW * 32, smem3_vp<QQ, NW, false>(), ctx->stream>>>(
                ctx->tmap[ctx->cur], args3<float>(ctx), consts3p<QQ, NC>(ctx));
    } else
        step3d<T, QQ, NC, NW><<<grid, NW * 32, smem3<T, QQ, NC, NW>(), ctx->stream>>>(args3<T>(ctx),
                                                                                      consts3<T, QQ, NC>(ctx));
    return cudaGetLastError();
}

// the step kernel for this context's precision, lattice and polynomial size
template <typename F>
auto dispatch3(const dugks_3d_ctx* ctx, F&& f) {
    if (ctx->precision == 32) {
        if (ctx->q == 19) return ctx->nc == 4 ? f.template operator()<float, 19, 4, 12>() : f.template operator()<float, 19, NCL, 12>();
        return ctx->nc == 4 ? f.template operator()<float, 15, 4, 12>() : f.template operator()<float, 15, NCL, 12>();
    }
    if (ctx->q == 19) return ctx->nc == 4 ? f.template operator()<double, 19, 4, 6>() : f.template operator()<double, 19, NCL, 6>();
    return ctx->nc == 4 ? f.template operator()<double, 15, 4, 6>() : f.template operator()<double, 15, NCL, 6>();
}

struct LaunchOp {
    dugks_3d_ctx* ctx;
    template <typename T, int QQ, int NC, int NW>
    cudaError_t operator()() const { return launch3<T, QQ, NC, NW>(ctx); }
};
struct AttrOp {
    template <typename T, int QQ, int NC, int NW>
    cudaError_t operator()() const {
        if constexpr (std::is_same<T, float>::value) {
            cudaError_t e;
            if constexpr (QQ == 15)
                e = cudaFuncSetAttribute(step3d_hv<QQ, NC, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem3_hv<QQ, NW>()));
            else
                e = cudaFuncSetAttribute(step3d_vp<QQ, NC, NW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem3_vp<QQ, NW, true>()));
            if (e != cudaSuccess) return e;
            return cudaFuncSetAttribute(step3d_vp<QQ, NC, NW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(smem3_vp<QQ, NW, false>()));
        } else
            return cudaFuncSetAttribute(step3d<T, QQ, NC, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(smem3<T, QQ, NC, NW>()));
    }
};
struct OccOp {
    int* occ;
    bool tma;
    template <typename T, int QQ, int NC, int NW>
    cudaError_t operator()() const {
        if constexpr (std::is_same<T, float>::value)
        {
            if (!tma)
                return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, step3d_vp<QQ, NC, NW, false>, NW * 32,
                                                                     smem3_vp<QQ, NW, false>());
            if constexpr (QQ == 15)
                return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, step3d_hv<QQ, NC, NW>, NW * 32,
                                                                     smem3_hv<QQ, NW>());
            else
                return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, step3d_vp<QQ, NC, NW, true>, NW * 32,
                                                                     smem3_vp<QQ, NW, true>());
        }
        else
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, step3d<T, QQ, NC, NW>, NW * 32,
                                                                 smem3<T, QQ, NC, NW>());
    }
};
struct NwOp {
    template <typename T, int QQ, int NC, int NW>
    int operator()() const { return NW; }
};
struct InitOp {
    dugks_3d_ctx* ctx;
    const void* phi0;
    template <typename T, int QQ, int NC, int NW>
    cudaError_t operator()() const {
        const long long n = (long long)ctx->nx * ctx->ny * ctx->nz;
        const int blocks = int(std::min<long long>((n + 255) / 256, 65535));
        init3<T, QQ, NC, T><<<blocks, 256, 0, ctx->stream>>>(static_cast<const T*>(phi0),
                                                            static_cast<T*>(ctx->buf[ctx->cur]), n,
                                                            consts3<T, QQ, NC>(ctx));
        return cudaGetLastError();
    }
};
struct PhiOp {
    dugks_3d_ctx* ctx;
    void* phi;
    template <typename T, int QQ, int NC, int NW>
    cudaError_t operator()() const {
        phi_mass3<T, QQ><<<ctx->red_blocks, 256, 0, ctx->stream>>>(
            static_cast<const T*>(ctx->buf[ctx->cur]), static_cast<T*>(phi), ctx->nx, ctx->ny, ctx->nz, ctx->width[0],
            ctx->width[1], ctx->width[2], ctx->partial);
        sum3<<<1, 256, 0, ctx->stream>>>(ctx->partial, ctx->red_blocks, ctx->mass_dev);
        return cudaGetLastError();
    }
};

void free3(dugks_3d_ctx* ctx) {
    if (!ctx) return;
    Guard3 g(ctx->device);
    for (void* p : {ctx->buf[0], ctx->buf[1], ctx->fm[0], ctx->fm[1], ctx->fm[2], ctx->cm[0], ctx->cm[1], ctx->cm[2],
                    static_cast<void*>(ctx->width[0]), static_cast<void*>(ctx->width[1]),
                    static_cast<void*>(ctx->width[2]), static_cast<void*>(ctx->partial),
                    static_cast<void*>(ctx->mass_dev), static_cast<void*>(ctx->err_dev)})
        if (p) cudaFree(p);
    delete ctx;
}

template <typename T>
cudaError_t upload_metrics(dugks_3d_ctx* ctx, const std::vector<double>* faces) {
    for (int d = 0; d < 3; ++d) {
        std::vector<FaceM<T>> fm;
        std::vector<CellM<T>> cm;
        std::vector<double> wd;
        metrics3<T>(faces[d], ctx->per[d] != 0, ctx->hc, ctx->dt, ctx->c, fm, cm, wd);
        cudaError_t e;
        if ((e = cudaMalloc(&ctx->fm[d], fm.size() * sizeof(fm[0]))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(ctx->fm[d], fm.data(), fm.size() * sizeof(fm[0]), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMalloc(&ctx->cm[d], cm.size() * sizeof(cm[0]))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(ctx->cm[d], cm.data(), cm.size() * sizeof(cm[0]), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMalloc(&ctx->width[d], wd.size() * sizeof(double))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(ctx->width[d], wd.data(), wd.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

dugks_status dugks_3d_check_config(const dugks_3d_mesh* mesh, const dugks_3d_vset* vset, const dugks_3d_coef* coef,
                                   double dt) {
    if (!mesh || !vset || !coef || !mesh->xf || !mesh->yf || !mesh->zf) return DUGKS_ERR_ARG;
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return DUGKS_ERR_ARG;
    if (mesh->nx > (1 << 20) || mesh->ny > (1 << 20) || mesh->nz > (1 << 20)) return DUGKS_ERR_ARG;
    if (vset->kind != DUGKS_D3Q15 && vset->kind != DUGKS_D3Q19) return DUGKS_ERR_ARG;
    if (coef->nb < 0 || coef->nb > 8 || coef->nd < 0 || coef->nd > 8) return DUGKS_ERR_ARG;
    for (int w = 0; w < 6; ++w)
        if (mesh->bc[w] != DUGKS_BC_PERIODIC && mesh->bc[w] != DUGKS_BC_DIRICHLET) return DUGKS_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if ((mesh->bc[2 * a] == DUGKS_BC_PERIODIC) != (mesh->bc[2 * a + 1] == DUGKS_BC_PERIODIC)) return DUGKS_ERR_ARG;
    const double* f[3] = {mesh->xf, mesh->yf, mesh->zf};
    const int n[3] = {mesh->nx, mesh->ny, mesh->nz};
    double hmin = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (!finite_n(f[a], n[a] + 1)) return DUGKS_ERR_CONFIG;
        for (int j = 0; j < n[a]; ++j) {
            const double w = f[a][j + 1] - f[a][j];
            if (!(w > 0.0)) return DUGKS_ERR_CONFIG;
            hmin = std::min(hmin, w);
        }
    }
    if (!finite_n(mesh->bc_value, 6) || !finite_n(coef->u, 3) || !finite_n(coef->b, coef->nb) ||
        !finite_n(coef->d, coef->nd) || !std::isfinite(coef->alpha) || !std::isfinite(vset->c) || !std::isfinite(dt))
        return DUGKS_ERR_CONFIG;
    if (!(vset->c > 0.0) || !(coef->alpha > 0.0) || !(dt > 0.0)) return DUGKS_ERR_CONFIG;
    if (!(vset->c * dt / hmin < 1.0)) return DUGKS_ERR_CONFIG;
    return DUGKS_OK;
}

dugks_status dugks_3d_create(const dugks_3d_mesh* mesh, const dugks_3d_vset* vset, const dugks_3d_coef* coef,
                             double dt, const dugks_options* opts, dugks_3d_ctx** out) {
    if (!out) return DUGKS_ERR_ARG;
    *out = nullptr;
    dugks_status st = dugks_3d_check_config(mesh, vset, coef, dt);
    if (st != DUGKS_OK) return st;
    dugks_options o = {DUGKS_FP32, DUGKS_KERNEL_FUSED, nullptr, -1};
    if (opts) o = *opts;
    if (o.precision != DUGKS_FP32 && o.precision != DUGKS_FP64) return DUGKS_ERR_ARG;
    if (o.kernel == DUGKS_KERNEL_NAIVE) return DUGKS_ERR_UNSUPPORTED;  // one 3-D kernel
    auto* ctx = new dugks_3d_ctx();
    if (o.device >= 0) ctx->device = o.device;
    else cudaGetDevice(&ctx->device);
    Guard3 guard(ctx->device);
    ctx->nx = mesh->nx; ctx->ny = mesh->ny; ctx->nz = mesh->nz;
    ctx->q = vset->kind;
    ctx->precision = o.precision;
    ctx->elem = o.precision == 32 ? sizeof(float) : sizeof(double);
    ctx->stream = static_cast<cudaStream_t>(o.stream);
    for (int a = 0; a < 3; ++a) ctx->per[a] = mesh->bc[2 * a] == DUGKS_BC_PERIODIC;
    for (int w = 0; w < 6; ++w) ctx->bcv[w] = mesh->bc_value[w];
    ctx->c = vset->c;
    ctx->dt = dt;
    // relaxation time from alpha = c_s^2 lambda (Section 3) and the weights of Eqs. 2.21, 2.22
    const double cs2 = vset->c * vset->c / 3.0, lam = coef->alpha / cs2, h = 0.5 * dt;
    ctx->lambda = lam;
    ctx->a_bp = (2.0 * lam - h) / (2.0 * lam + dt);
    ctx->b_bp = 3.0 * h / (2.0 * lam + dt);
    ctx->a_f = 2.0 * lam / (2.0 * lam + h);
    ctx->b_f = h / (2.0 * lam + h);
    ctx->hc = h * vset->c;
    // Eq. 2.3 per velocity as a polynomial in phi (e_i the unit direction, |e|^2 in 0..3):
    //   feq_i = w_i [ phi + 3 (e.u)/c b + 3 (|e|^2 - 1)/2 (d - phi) + (9 (e.u)^2 - 3 |u|^2)/(2 c^2) Cint ]
    double cint[NCL] = {0};
    if (!coef->c_zero)
        for (int kq = 1; kq < coef->nb; ++kq)
            for (int l = 1; l < coef->nb; ++l) cint[kq + l - 1] += double(kq) * l * coef->b[kq] * coef->b[l] / (kq + l - 1);
    const double u2 = coef->u[0] * coef->u[0] + coef->u[1] * coef->u[1] + coef->u[2] * coef->u[2];
    int maxdeg = 1;
    for (int i = 0; i < ctx->q; ++i) {
        const double eu = dir3(ctx->q, i, 0) * coef->u[0] + dir3(ctx->q, i, 1) * coef->u[1] + dir3(ctx->q, i, 2) * coef->u[2];
        double e2 = 0;
        for (int a = 0; a < 3; ++a) e2 += dir3(ctx->q, i, a) * dir3(ctx->q, i, a);
        const double kb = 3.0 * eu / vset->c, kd = 3.0 * (e2 - 1.0) / 2.0;
        const double kc = (9.0 * eu * eu - 3.0 * u2) / (2.0 * vset->c * vset->c);
        for (int m = 0; m < NCL; ++m) {
            const double bm = m < coef->nb ? coef->b[m] : 0.0, dm = m < coef->nd ? coef->d[m] : 0.0;
            const double one = m == 1 ? 1.0 : 0.0;
            const double v = weight3(ctx->q, i) * (one + kb * bm + kd * (dm - one) + kc * cint[m]);
            ctx->feq_coef[i][m] = v;
            if (v != 0.0) maxdeg = std::max(maxdeg, m);
        }
    }
    ctx->nc = maxdeg <= 3 ? 4 : NCL;
    double hmin = INFINITY;
    std::vector<double> faces[3] = {std::vector<double>(mesh->xf, mesh->xf + mesh->nx + 1),
                                    std::vector<double>(mesh->yf, mesh->yf + mesh->ny + 1),
                                    std::vector<double>(mesh->zf, mesh->zf + mesh->nz + 1)};
    for (int a = 0; a < 3; ++a)
        for (size_t j = 0; j + 1 < faces[a].size(); ++j) hmin = std::min(hmin, faces[a][j + 1] - faces[a][j]);
    ctx->cfl = vset->c * dt / hmin;

    const size_t bytes = size_t(ctx->q) * ctx->nx * ctx->ny * ctx->nz * ctx->elem;
    cudaError_t e;
    for (int b = 0; b < 2; ++b) {
        if ((e = cudaMalloc(&ctx->buf[b], bytes)) != cudaSuccess) { st = fail3(ctx, e, "cudaMalloc(state)"); free3(ctx); return st; }
        if ((e = cudaMemsetAsync(ctx->buf[b], 0, bytes, ctx->stream)) != cudaSuccess) { st = fail3(ctx, e, "cudaMemsetAsync"); free3(ctx); return st; }
    }
    e = ctx->precision == 32 ? upload_metrics<float>(ctx, faces) : upload_metrics<double>(ctx, faces);
    if (e != cudaSuccess) { st = fail3(ctx, e, "metrics"); free3(ctx); return st; }
    const long long cells = (long long)ctx->nx * ctx->ny * ctx->nz;
    ctx->red_blocks = int(std::min<long long>((cells + 255) / 256, 2048));
    if ((e = cudaMalloc(&ctx->partial, sizeof(double) * ctx->red_blocks)) != cudaSuccess ||
        (e = cudaMalloc(&ctx->mass_dev, sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->err_dev, sizeof(int))) != cudaSuccess ||
        (e = cudaMemsetAsync(ctx->err_dev, 0, sizeof(int), ctx->stream)) != cudaSuccess) {
        st = fail3(ctx, e, "cudaMalloc(reduction)");
        free3(ctx);
        return st;
    }
    if ((e = dispatch3(ctx, AttrOp{})) != cudaSuccess) { st = fail3(ctx, e, "cudaFuncSetAttribute"); free3(ctx); return st; }
    // FP32 with nx a multiple of 4 (the TMA box origin) and the Q planes below 2^32 elements (the
    // TMA kernels address them by 32-bit offsets): ftilde staged by TMA boxes, D3Q19 in step3d_vp
    // (256^3: 1132 us against 1269 us with per-thread cp.async copies), D3Q15 in the face-halves
    // kernel step3d_hv (1166 us; step3d_vp 1214 with cp.async, 1275 with TMA); otherwise step3d_vp
    // with cp.async copies and 64-bit offsets
    const long long elems = (long long)ctx->q * ctx->nx * ctx->ny * ctx->nz;
    ctx->tma = ctx->precision == 32 && ctx->nx % 4 == 0 && elems < (1ll << 32) && encode_tmaps3(ctx);
    // grid: 30-column strips x (NW-2)-row blocks x z segments.  The segment length
    // minimises (waves of resident CTAs) x (planes per CTA + about one plane of
    // pipeline fill), with segments of at least 8 planes where nz allows.
    ctx->nw = dispatch3(ctx, NwOp{});
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if ((e = dispatch3(ctx, OccOp{&occ, ctx->tma})) != cudaSuccess || occ < 1) {
        st = e != cudaSuccess ? fail3(ctx, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor") : DUGKS_ERR_UNSUPPORTED;
        if (occ < 1 && e == cudaSuccess) ctx->last_error = "the 3-D step kernel does not fit on an SM";
        free3(ctx);
        return st;
    }
    ctx->grid[0] = (ctx->nx + 29) / 30;
    ctx->grid[1] = (ctx->ny + ctx->nw - 3) / (ctx->nw - 2);
    const long long tiles = (long long)ctx->grid[0] * ctx->grid[1];
    const long long slots = (long long)std::max(sms, 1) * occ;
    double best = INFINITY;
    for (int zs = ctx->nz; zs >= std::min(8, ctx->nz); --zs) {
        const long long nseg = (ctx->nz + zs - 1) / zs;
        if (nseg > 65535) break;
        const double cost = double((tiles * nseg + slots - 1) / slots) * (zs + 1.0);
        if (cost < best * (1.0 - 1e-9)) {
            best = cost;
            ctx->zseg = zs;
        }
    }
    ctx->grid[2] = (ctx->nz + ctx->zseg - 1) / ctx->zseg;
    if (ctx->grid[1] > 65535) { free3(ctx); return DUGKS_ERR_ARG; }
    *out = ctx;
    return DUGKS_OK;
}

dugks_status dugks_3d_destroy(dugks_3d_ctx* ctx) {
    if (!ctx) return DUGKS_OK;
    {
        Guard3 g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
    }
    free3(ctx);
    return DUGKS_OK;
}

dugks_status dugks_3d_init_phi(dugks_3d_ctx* ctx, const void* phi0_dev) {
    if (!ctx || !phi0_dev) return DUGKS_ERR_ARG;
    Guard3 g(ctx->device);
    CK3(dispatch3(ctx, InitOp{ctx, phi0_dev}));
    ctx->steps_done = 0;
    return DUGKS_OK;
}

dugks_status dugks_3d_step(dugks_3d_ctx* ctx, long long n) {
    if (!ctx || n < 0) return DUGKS_ERR_ARG;
    Guard3 g(ctx->device);
    for (long long s = 0; s < n; ++s) {
        CK3(dispatch3(ctx, LaunchOp{ctx}));
        ctx->cur ^= 1;
        ++ctx->steps_done;
    }
    return DUGKS_OK;
}

dugks_status dugks_3d_get_phi(dugks_3d_ctx* ctx, void* phi_dev_out, double* mass_out) {
    if (!ctx) return DUGKS_ERR_ARG;
    Guard3 g(ctx->device);
    CK3(dispatch3(ctx, PhiOp{ctx, phi_dev_out}));
    if (mass_out) {
        CK3(cudaMemcpyAsync(mass_out, ctx->mass_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK3(cudaStreamSynchronize(ctx->stream));
        if (!std::isfinite(*mass_out)) return DUGKS_ERR_NONFINITE;
    }
    return DUGKS_OK;
}

dugks_status dugks_3d_save_state(dugks_3d_ctx* ctx, void* f_dev_out) {
    if (!ctx || !f_dev_out) return DUGKS_ERR_ARG;
    Guard3 g(ctx->device);
    const size_t bytes = size_t(ctx->q) * ctx->nx * ctx->ny * ctx->nz * ctx->elem;
    CK3(cudaMemcpyAsync(f_dev_out, ctx->buf[ctx->cur], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    return DUGKS_OK;
}

dugks_status dugks_3d_load_state(dugks_3d_ctx* ctx, const void* f_dev_in) {
    if (!ctx || !f_dev_in) return DUGKS_ERR_ARG;
    Guard3 g(ctx->device);
    const size_t bytes = size_t(ctx->q) * ctx->nx * ctx->ny * ctx->nz * ctx->elem;
    CK3(cudaMemcpyAsync(ctx->buf[ctx->cur], f_dev_in, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->steps_done = 0;
    return DUGKS_OK;
}

dugks_status dugks_3d_sync(dugks_3d_ctx* ctx) {
    if (!ctx) return DUGKS_ERR_ARG;
    Guard3 g(ctx->device);
    CK3(cudaStreamSynchronize(ctx->stream));
    CK3(cudaGetLastError());
    int err = 0;
    CK3(cudaMemcpy(&err, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        CK3(cudaMemset(ctx->err_dev, 0, sizeof(int)));
        ctx->last_error = "a bounded TMA wait in the 3-D step expired";
        return DUGKS_ERR_TIMEOUT;
    }
    return DUGKS_OK;
}

dugks_status dugks_3d_info(const dugks_3d_ctx* ctx, dugks_3d_info_t* out) {
    if (!ctx || !out) return DUGKS_ERR_ARG;
    out->nx = ctx->nx; out->ny = ctx->ny; out->nz = ctx->nz;
    out->q = ctx->q;
    out->precision = ctx->precision;
    out->steps_done = ctx->steps_done;
    out->dt = ctx->dt;
    out->lambda = ctx->lambda;
    out->cfl = ctx->cfl;
    out->block_threads = ctx->nw * 32;
    for (int d = 0; d < 3; ++d) out->grid[d] = ctx->grid[d];
    out->zseg = ctx->zseg;
    out->state_bytes = (long long)ctx->q * ctx->nx * ctx->ny * ctx->nz * (long long)ctx->elem;
    return DUGKS_OK;
}

const char* dugks_3d_last_error(const dugks_3d_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

}  // extern "C"
