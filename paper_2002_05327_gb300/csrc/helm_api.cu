// libhelm host side: problem setup, scheduling of Algorithm 3.1 / 4.1 by
// dependency levels, the factor driver, the DDM application, FP64 flexible
// GMRES (Remark 1), the adjoint and the C ABI of include/helm.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <functional>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "helm_internal.h"

using namespace helm;
using cd = std::complex<double>;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? HELM_ERR_OOM : HELM_ERR_CUDA,       \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

#define TRY(call)                  \
    do {                           \
        int r_ = (call);           \
        if (r_ != HELM_OK) return r_; \
    } while (0)

// ----------------------------------------------------------------------------- PML profile
// sigma at cell position p for one side: the PML starts `gap` cells beyond
// `face` and is `width` cells thick (Eq. 2.1; Eq. 2.3 for gap = d).
struct SideP {
    double face, gap, width;
};
struct AxisP {
    int lo, hi;
    SideP left, right;
};

double sigma_at(double p, const AxisP& ax, double sigma0, int power) {
    double s = 0.0;
    double tl = ax.left.face - p;
    if (tl > ax.left.gap) s += sigma0 * std::pow((tl - ax.left.gap) / ax.left.width, power);
    double tr = p - ax.right.face;
    if (tr > ax.right.gap) s += sigma0 * std::pow((tr - ax.right.gap) / ax.right.width, power);
    return s;
}

cd alpha_at(double p, const AxisP& ax, const helm_pml& pml, double omega) {
    double s = sigma_at(p, ax, pml.sigma0, pml.power);
    if (pml.form == HELM_PML_OMEGA) s /= omega;
    return cd(1.0, s);
}

// beta_hat(t) = 1 - (10 t^3 - 15 t^4 + 6 t^5) on [0,1]: a monotone C^2 cutoff.
double beta_hat(double t) {
    if (t <= 0) return 1.0;
    if (t >= 1) return 0.0;
    return 1.0 - t * t * t * (10.0 - 15.0 * t + 6.0 * t * t);
}

}  // namespace

// ----------------------------------------------------------------------------- context
struct helm_ctx {
    DevProblem P{};
    int64_t n[3]{};
    helm_pml pml{};
    int W = 0;
    helm_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cstream = nullptr;  // host <-> device copies of chunked solves (created on first use)
    int device = -1;                   // the device current at helm_setup
    int prec = HELM_PREC_MIXED;
    int nsweeps = 0;

    std::vector<SubDesc> subs_h;
    SubDesc* subs_d = nullptr;
    int nbp_max = 0;

    // global problem
    cplx<double>* g_alpha = nullptr;  // per axis: nodes then faces
    Win<double> gwin{};
    float4* stc_d = nullptr;           // per node: the J-multiplied stencil, float-float
    double* m64 = nullptr;
    float* m32 = nullptr;
    int64_t Ng = 0;

    // subdomain coefficients (double and float copies)
    cplx<double>* an64 = nullptr;
    cplx<double>* af64 = nullptr;
    cplx<float>* an32 = nullptr;
    cplx<float>* af32 = nullptr;
    cplx<double>* Pv64 = nullptr;
    cplx<double>* inva64 = nullptr;
    cplx<float>* Pv32 = nullptr;
    cplx<float>* inva32 = nullptr;
    double* tab64 = nullptr;
    float* tab32 = nullptr;
    int* box_of = nullptr;

    // factors
    void* ufac = nullptr;              // tcgen05 tile image of the factors (TF32)
    size_t ufac_bytes = 0;
    int64_t* ufac_off = nullptr;       // byte offset per subdomain
    int umma_mt = 0;                   // CTAs per block in the tcgen05 solve (0: not used)
    int umma_nblk = 0;                 // largest block of the tcgen05 solve
    int umma_lines = 0;                // most lines of a subdomain (twisted solve)
    bool umma_twist = false;           // tcgen05 solve in its twisted (two-ended) form
    std::map<int, int> panel_pick;     // nrhs -> measured right-hand sides per CTA (tune_panel)
    bool f16 = false;                  // HELM_PREC_F16: FP16 operands in the twisted solve
    int* ascale_d = nullptr;           // per (subdomain, line) exponent of the FP16 factor scale
    void* bsrc = nullptr;              // local sources b, same layout as buf; zero except where the
                                       // gather writes (sweep-0 boxes, transfer strips)
    size_t inva_count = 0;             // entries of inva (nlines + 1 per subdomain)
    void* fac = nullptr;
    size_t fac_bytes = 0;
    bool factored = false;
    double t_factor_ms = 0;
    int* err_d = nullptr;
    uint32_t wait_polls = kDefaultWaitPolls;  // ordinary bounded waits of the solve kernels

    // schedule
    std::vector<std::vector<Task>> levels;
    std::vector<int> level_off;
    Task* tasks_d = nullptr;
    Incoming* inc_d = nullptr;
    GNode* gnode_d = nullptr;          // gather work list (nodes)
    GBlock* gblk_d = nullptr;          // gather work list (blocks, level after level)
    std::vector<int> gblk_off;         // first block of each level, and the total
    std::vector<int64_t> gnodes_lv;    // work-list nodes per level
    std::vector<int64_t> node_buf_h;  // (l*nsub + s) -> element offset, or -1 if inactive
    int64_t* node_buf_d = nullptr;
    int64_t buf_per_rhs = 0;
    int nsolves = 0;

    // work buffers
    int cap_rhs = 0;
    void* buf = nullptr;           // window buffers, complex T, [rhs][nodes][window]
    cplx<double>* bvec = nullptr;  // J-scaled source of one DDM application
    int cap_vec_rhs = 0;
    std::vector<cplx<double>*> gm;  // GMRES vectors (each nrhs*Ng entries of 16 bytes; float-float)
    int gm_rhs = 0;
    cplx<double>* stage_d[3] = {};     // device staging of the caller's host arrays (grow-only)
    size_t stage_cap[3] = {};
    float4** vptr_d = nullptr;  // device copies of the V_i and Z_i pointers
    float4** zptr_d = nullptr;
    cplx<double>* small_d = nullptr;  // dots / coefficients
    cplx<double>* partial_d = nullptr;
    size_t small_cap = 0;
    size_t dev_bytes = 0;

    // profiling: per class counters and pending event pairs
    helm_profile prof{};
    struct Pending {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

// Every device allocation of a context goes through here: it is refused with
// HELM_ERR_OOM (before cudaMalloc is called) when it would take the context's
// device bytes beyond cfg.max_device_bytes, if that is set.
int ctx_malloc(helm_ctx* c, void** p, size_t bytes) {
    const size_t cap = c->cfg.max_device_bytes > 0 ? (size_t)c->cfg.max_device_bytes : 0;
    if (cap && c->dev_bytes + bytes > cap)
        return fail(HELM_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes beyond the context's cap of " +
                                      std::to_string(cap) + " bytes (" + std::to_string(c->dev_bytes) + " in use)");
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? HELM_ERR_OOM : HELM_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return HELM_OK;
}
#define CKM(ptr, bytes) TRY(ctx_malloc(c, (void**)(ptr), (bytes)))

size_t elem_size(const helm_ctx* c) { return c->prec == HELM_PREC_F64 ? 16 : 8; }

cudaEvent_t pool_event(helm_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket `launches` kernel launches of class cls with CUDA events on the
// context's stream (when profiling) and count them.
struct ProfScope {
    helm_ctx* c;
    int cls;
    cudaEvent_t b = nullptr;
    ProfScope(helm_ctx* c_, int cls_, int launches, double bytes = 0, double flops = 0)
        : c(c_), cls(cls_) {
        c->prof.launches[cls] += launches;
        c->prof.bytes[cls] += bytes;
        c->prof.flops[cls] += flops;
        if (c->cfg.profile) {
            b = pool_event(c);
            cudaEventRecord(b, c->stream);
        }
    }
    ~ProfScope() {
        if (c->cfg.profile) {
            cudaEvent_t e = pool_event(c);
            cudaEventRecord(e, c->stream);
            c->pending.push_back({cls, b, e});
        }
    }
};

// Resolve pending event pairs (the stream must be synchronised).
void resolve_profile(helm_ctx* c) {
    for (auto& p : c->pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->prof.ms[p.cls] += ms;
        c->event_pool.push_back(p.a);
        c->event_pool.push_back(p.b);
    }
    c->pending.clear();
}

int ensure_buffers(helm_ctx* c, int nrhs) {
    if (nrhs <= c->cap_rhs && c->buf) return HELM_OK;
    if (c->buf) {
        cudaFree(c->buf);
        cudaFree(c->bsrc);
        c->dev_bytes -= 2 * (size_t)c->cap_rhs * c->buf_per_rhs * elem_size(c);
        c->buf = c->bsrc = nullptr;
    }
    size_t bytes = (size_t)nrhs * c->buf_per_rhs * elem_size(c);
    CKM(&c->buf, bytes);
    CKM(&c->bsrc, bytes);
    CK(cudaMemsetAsync(c->bsrc, 0, bytes, c->stream));  // the gather writes only its fixed node set
    c->dev_bytes += 2 * bytes;
    c->cap_rhs = nrhs;
    return HELM_OK;
}

int ensure_bvec(helm_ctx* c, int nrhs) {
    if (nrhs <= c->cap_vec_rhs && c->bvec) return HELM_OK;
    if (c->bvec) {
        cudaFree(c->bvec);
        c->dev_bytes -= (size_t)c->cap_vec_rhs * c->Ng * 16;
        c->bvec = nullptr;
    }
    CKM(&c->bvec, (size_t)nrhs * c->Ng * 16);
    c->dev_bytes += (size_t)nrhs * c->Ng * 16;
    c->cap_vec_rhs = nrhs;
    return HELM_OK;
}

int ensure_small(helm_ctx* c, size_t count) {
    if (count <= c->small_cap) return HELM_OK;
    if (c->small_d) cudaFree(c->small_d);
    if (c->partial_d) cudaFree(c->partial_d);
    CKM(&c->small_d, count * sizeof(cplx<double>));
    CKM(&c->partial_d, count * 256 * sizeof(cplx<double>));  // <= 256 block partials per output
    if (!c->vptr_d) {
        CKM(&c->vptr_d, 64 * sizeof(void*));
        CKM(&c->zptr_d, 64 * sizeof(void*));
    }
    c->small_cap = count;
    return HELM_OK;
}

// ----------------------------------------------------------------------------- routing (Rules 3.1/3.2, 4.1/4.2)
// Sweep order: in 2D (+,+), (-,+), (+,-), (-,-) (Algorithm 3.1); in 3D the
// list (Sorder3D) of Algorithm 4.1 (x flips fastest, then y, then z), or with
// order 1 the alternative of Section 4.1 whose L1 distance to the first
// direction never decreases.
std::vector<std::array<int, 3>> sweep_dirs(int ndim, int order) {
    std::vector<std::array<int, 3>> S;
    for (int l = 0; l < (1 << ndim); ++l) {
        std::array<int, 3> D{0, 0, 0};
        for (int a = 0; a < ndim; ++a) D[a] = ((l >> a) & 1) ? -1 : 1;
        S.push_back(D);
    }
    if (ndim == 3 && order == 1)
        S = {{{1, 1, 1}}, {{-1, 1, 1}}, {{1, -1, 1}}, {{1, 1, -1}},
             {{-1, -1, 1}}, {{-1, 1, -1}}, {{1, -1, -1}}, {{-1, -1, -1}}};
    return S;
}

std::vector<std::array<int, 3>> transfer_dirs(int ndim) {
    std::vector<std::array<int, 3>> out;
    for (int dz = (ndim == 3 ? 1 : 0); dz >= (ndim == 3 ? -1 : 0); --dz)
        for (int dy = 1; dy >= -1; --dy)
            for (int dx = 1; dx >= -1; --dx)
                if (dx || dy || dz) out.push_back({dx, dy, dz});
    return out;
}

// Rule 3.1 (2D): d.D > 0.  Rule 4.1 (3D): d.D > 0 and d(k) D(k) >= 0 for all k.
bool similar(const std::array<int, 3>& d, const std::array<int, 3>& D, int ndim) {
    int dot = 0;
    bool nonneg = true;
    for (int a = 0; a < ndim; ++a) {
        dot += d[a] * D[a];
        nonneg &= d[a] * D[a] >= 0;
    }
    return ndim == 2 ? dot > 0 : (dot > 0 && nonneg);
}

// Rule 3.2 / 4.2: not used in a later sweep if in some coordinate plane the
// projection of the source direction has exactly one zero and the projected
// generating and using sweep directions are opposite.
bool blocked(const std::array<int, 3>& d, const std::array<int, 3>& Dg,
             const std::array<int, 3>& Du, int ndim) {
    const int planes2[1][2] = {{0, 1}};
    const int planes3[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    int np = ndim == 2 ? 1 : 3;
    for (int i = 0; i < np; ++i) {
        int a = ndim == 2 ? planes2[i][0] : planes3[i][0];
        int b = ndim == 2 ? planes2[i][1] : planes3[i][1];
        int zeros = (d[a] == 0) + (d[b] == 0);
        if (zeros == 1 && Dg[a] == -Du[a] && Dg[b] == -Du[b]) return true;
    }
    return false;
}

int route_of(int l, const std::array<int, 3>& d, const std::vector<std::array<int, 3>>& S, int ndim) {
    for (int l2 = l; l2 < (int)S.size(); ++l2)
        if (similar(d, S[l2], ndim) && !blocked(d, S[l], S[l2], ndim)) return l2;
    return -1;
}

void fill_window_alpha(const AxisP& ax, const helm_pml& pml, double omega, std::vector<cd>& nodes,
                       std::vector<cd>& faces) {
    for (int k = ax.lo; k < ax.hi; ++k) nodes.push_back(alpha_at(k + 0.5, ax, pml, omega));
    for (int k = ax.lo; k <= ax.hi; ++k) faces.push_back(alpha_at((double)k, ax, pml, omega));
}

template <typename T>
int upload(T** dst, const void* src, size_t bytes, helm_ctx* c) {
    CKM(dst, bytes);
    if (bytes) CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    c->dev_bytes += bytes;
    return HELM_OK;
}

// Gather work list (k_transfer.cu): per task, in level order, the window
// nodes the first sweep's box or an incoming transfer's strip reaches.  A
// strip is a box of nodes: along each axis the transfer points through, the
// d + 1 nodes beyond the sender's box face (the receiver evaluates
// -A_recv(beta v) there; beta vanishes from the d-th node on and its residual
// reaches one node further); along the other axes, the whole window.
int build_gather_list(helm_ctx* c, const std::vector<Task>& tasks, const std::vector<Incoming>& inc) {
    const int ndim = c->P.ndim, d = c->P.d;
    std::vector<GNode> nodes;
    std::vector<GBlock> blocks;
    std::vector<uint32_t> mark;
    c->gblk_off.clear();
    c->gnodes_lv.clear();
    for (size_t lv = 0; lv + 1 < c->level_off.size(); ++lv) {
        c->gblk_off.push_back((int)blocks.size());
        const int64_t lv_first = (int64_t)nodes.size();
        for (int ti = c->level_off[lv]; ti < c->level_off[lv + 1]; ++ti) {
            const Task& t = tasks[ti];
            const SubDesc& S = c->subs_h[t.sub];
            mark.assign((size_t)S.win_elems, 0u);
            // global node ranges [lo, hi), clipped to the receiver's window
            auto paint = [&](const int lo[3], const int hi[3], uint32_t bit) {
                int a0[3], a1[3];
                for (int a = 0; a < 3; ++a) {
                    a0[a] = std::max(lo[a], S.lo[a]) - S.lo[a];
                    a1[a] = std::min(hi[a], S.hi[a]) - S.lo[a];
                    if (a0[a] >= a1[a]) return;
                }
                for (int z = a0[2]; z < a1[2]; ++z)
                    for (int y = a0[1]; y < a1[1]; ++y)
                        for (int x = a0[0]; x < a1[0]; ++x)
                            mark[((size_t)z * S.nw[1] + y) * S.nw[0] + x] |= bit;
            };
            if (t.sweep == 0) paint(S.box_lo, S.box_hi, 1u << 31);
            for (int i = 0; i < t.in_cnt; ++i) {
                const Incoming& I = inc[(size_t)t.in_off + i];
                const SubDesc& R = c->subs_h[I.sender];
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    lo[a] = S.lo[a];
                    hi[a] = S.hi[a];
                    if (a >= ndim) continue;
                    if (I.dir[a] > 0) {
                        lo[a] = R.box_hi[a];
                        hi[a] = R.box_hi[a] + d + 1;
                    } else if (I.dir[a] < 0) {
                        lo[a] = R.box_lo[a] - 1 - d;
                        hi[a] = R.box_lo[a];
                    }
                }
                paint(lo, hi, 1u << i);
            }
            const int64_t first = (int64_t)nodes.size();
            for (size_t k = 0; k < mark.size(); ++k)
                if (mark[k]) nodes.push_back({(uint32_t)k, mark[k]});
            for (int64_t n0 = first; n0 < (int64_t)nodes.size(); n0 += kGB)
                blocks.push_back({ti, (int)std::min<int64_t>(kGB, (int64_t)nodes.size() - n0), n0});
        }
        c->gnodes_lv.push_back((int64_t)nodes.size() - lv_first);
    }
    c->gblk_off.push_back((int)blocks.size());
    TRY(upload(&c->gnode_d, nodes.data(), nodes.size() * sizeof(GNode), c));
    TRY(upload(&c->gblk_d, blocks.data(), blocks.size() * sizeof(GBlock), c));
    return HELM_OK;
}

std::vector<cplx<double>> to_c128(const std::vector<cd>& v) {
    std::vector<cplx<double>> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = {v[i].real(), v[i].imag()};
    return o;
}
std::vector<cplx<float>> to_c64(const std::vector<cd>& v) {
    std::vector<cplx<float>> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = {(float)v[i].real(), (float)v[i].imag()};
    return o;
}

int setup_impl(helm_ctx* c, int ndim, const int64_t n[3], double h, double omega, const double* m,
               const helm_pml* pml, const helm_partition* part, const helm_config* cfg) {
    if (ndim != 2 && ndim != 3) return fail(HELM_ERR_ARG, "ndim must be 2 or 3");
    if (!n || !m || !pml || !part) return fail(HELM_ERR_ARG, "null argument");
    if (!(h > 0) || !(omega > 0)) return fail(HELM_ERR_ARG, "h and omega must be positive");
    if (pml->width < 1 || pml->power < 0 || !(pml->sigma0 >= 0))
        return fail(HELM_ERR_ARG, "invalid PML");
    if (part->overlap < 1 || part->overlap > 128) return fail(HELM_ERR_ARG, "overlap must be in 1..128");
    if (cfg) c->cfg = *cfg;
    c->prec = HELM_PREC_MIXED;
    if (cfg && (cfg->precision == HELM_PREC_F64 || cfg->precision == HELM_PREC_TF32))
        c->prec = cfg->precision;
    if (cfg && cfg->precision == HELM_PREC_F16) {  // TF32 everywhere else, FP16 in the twisted solve
        c->prec = HELM_PREC_TF32;
        c->f16 = true;
    }
    if (c->cfg.restart <= 0) c->cfg.restart = 30;
    if (c->cfg.restart > 63) return fail(HELM_ERR_ARG, "restart must be at most 63");
    if (c->cfg.wait_limit < -1) return fail(HELM_ERR_ARG, "wait_limit must be -1, 0 or positive");
    if (c->cfg.sweep_order != 0 && c->cfg.sweep_order != 1) return fail(HELM_ERR_ARG, "sweep_order must be 0 or 1");
    if (c->cfg.algorithm != 0 && c->cfg.algorithm != 1) return fail(HELM_ERR_ARG, "algorithm must be 0 or 1");
    c->wait_polls = c->cfg.wait_limit == 0    ? kDefaultWaitPolls
                    : c->cfg.wait_limit == -1 ? 0u
                                              : (uint32_t)c->cfg.wait_limit;
    c->pml = *pml;
    c->W = part->sub_pml > 0 ? part->sub_pml : pml->width;
    DevProblem& P = c->P;
    P.ndim = ndim;
    P.h = h;
    P.omega = omega;
    P.d = part->overlap;
    const int Wg = pml->width;
    for (int a = 0; a < 3; ++a) {
        c->n[a] = a < ndim ? n[a] : 1;
        if (a < ndim && (n[a] < 1 || n[a] > (1 << 20))) return fail(HELM_ERR_ARG, "bad grid size");
        P.N[a] = a < ndim ? (int)(n[a] + 2 * Wg) : 1;
        P.nb[a] = a < ndim ? part->nb[a] : 1;
        if (a < ndim && (P.nb[a] < 1 || P.nb[a] > 4096)) return fail(HELM_ERR_ARG, "bad nb");
    }
    c->Ng = (int64_t)P.N[0] * P.N[1] * P.N[2];
    P.nsub = P.nb[0] * P.nb[1] * P.nb[2];
    // diagonal sweeps: 2^n sweeps; additive (Algorithm 2.1/2.2): one "sweep" index per step
    c->nsweeps = c->cfg.algorithm == 1 ? P.nb[0] + P.nb[1] + P.nb[2] - 3 + 1 : 1 << ndim;
    // host-side checks before any device work: the medium, and the device-memory cap
    // against the grid arrays setup allocates (m in float64 and float32, the stencil)
    for (int64_t i = 0; i < c->Ng; ++i)
        if (!std::isfinite(m[i]))
            return fail(HELM_ERR_NUMERIC, "m has a non-finite value at full-grid index " + std::to_string(i));
    if (c->cfg.max_device_bytes < 0) return fail(HELM_ERR_ARG, "max_device_bytes must be >= 0");
    {
        const double grid_bytes = (double)c->Ng * (8.0 + 4.0 + (1 + 2 * ndim) * 16.0);
        if (c->cfg.max_device_bytes > 0 && grid_bytes > (double)c->cfg.max_device_bytes)
            return fail(HELM_ERR_OOM, "the grid arrays need " + std::to_string((int64_t)grid_bytes) +
                                          " bytes, beyond the context's cap of " +
                                          std::to_string(c->cfg.max_device_bytes) + " bytes");
    }

    // ---- boxes per axis (global node ranges); edge boxes run over the global PML.
    // Host only, before any device work, so that a bad partition is refused first.
    std::vector<std::vector<int>> blo(3), bhi(3);
    for (int a = 0; a < 3; ++a) {
        if (a >= ndim) {
            blo[a] = {0};
            bhi[a] = {1};
            continue;
        }
        std::vector<int64_t> cut(P.nb[a] + 1);
        if (part->cuts[a]) {
            for (int i = 0; i <= P.nb[a]; ++i) cut[i] = part->cuts[a][i];
            if (cut[0] != 0 || cut[P.nb[a]] != c->n[a]) return fail(HELM_ERR_ARG, "cuts must span 0..n");
        } else {
            for (int i = 0; i <= P.nb[a]; ++i) cut[i] = (i * c->n[a]) / P.nb[a];
        }
        for (int i = 0; i < P.nb[a]; ++i) {
            if (cut[i + 1] <= cut[i]) return fail(HELM_ERR_ARG, "cuts must increase");
            blo[a].push_back(i == 0 ? 0 : (int)(Wg + cut[i]));
            bhi[a].push_back(i == P.nb[a] - 1 ? P.N[a] : (int)(Wg + cut[i + 1]));
            if (bhi[a].back() - blo[a].back() < P.d + 2)
                return fail(HELM_ERR_ARG, "box narrower than overlap + 2");
            // 3D: an inner box at least 2d wide, so that the cutoffs of at most
            // one neighbour per axis reach a node and the assembly's list of
            // eight boxes per node holds them all
            if (ndim == 3 && i > 0 && i + 1 < P.nb[a] && bhi[a].back() - blo[a].back() < 2 * P.d)
                return fail(HELM_ERR_ARG, "3D inner box narrower than twice the overlap");
        }
    }

    CK(cudaGetDevice(&c->device));
    if (c->cfg.stream) {
        c->stream = (cudaStream_t)c->cfg.stream;
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }

    // ---- global alphas
    std::vector<AxisP> gax(3);
    std::vector<cd> gall;
    int64_t goff[3][2];
    for (int a = 0; a < 3; ++a) {
        AxisP ax{0, P.N[a], {(double)Wg, 0.0, (double)Wg}, {(double)(Wg + c->n[a]), 0.0, (double)Wg}};
        gax[a] = ax;
        std::vector<cd> nodes, faces;
        if (a < ndim) fill_window_alpha(ax, *pml, omega, nodes, faces);
        else {
            nodes.assign(1, cd(1, 0));
            faces.assign(2, cd(1, 0));
        }
        goff[a][0] = gall.size();
        gall.insert(gall.end(), nodes.begin(), nodes.end());
        goff[a][1] = gall.size();
        gall.insert(gall.end(), faces.begin(), faces.end());
    }
    auto g128 = to_c128(gall);
    TRY(upload(&c->g_alpha, g128.data(), g128.size() * sizeof(cplx<double>), c));
    for (int a = 0; a < 3; ++a) {
        c->gwin.lo[a] = 0;
        c->gwin.n[a] = P.N[a];
        c->gwin.alpha_node[a] = c->g_alpha + goff[a][0];
        c->gwin.alpha_face[a] = c->g_alpha + goff[a][1];
    }
    // ---- medium
    TRY(upload(&c->m64, m, c->Ng * sizeof(double), c));
    {
        std::vector<float> m32(c->Ng);
        for (int64_t i = 0; i < c->Ng; ++i) m32[i] = (float)m[i];
        TRY(upload(&c->m32, m32.data(), c->Ng * sizeof(float), c));
    }
    // ---- the global operator's stencil, once (operator products, residuals)
    {
        const size_t bytes = (size_t)c->Ng * (1 + 2 * ndim) * sizeof(float4);
        CKM(&c->stc_d, bytes);
        c->dev_bytes += bytes;
        launch_stencil_ff(P, c->gwin, c->m64, c->stc_d, c->stream);
        CK(cudaGetLastError());
    }
    std::vector<int> box_of;
    for (int a = 0; a < ndim; ++a)
        for (int k = 0; k < P.N[a]; ++k) {
            int i = 0;
            while (k >= bhi[a][i]) ++i;
            box_of.push_back(i);
        }
    TRY(upload(&c->box_of, box_of.data(), box_of.size() * sizeof(int), c));

    // ---- subdomain windows and their coefficients
    std::vector<cd> an, af, pv, ia;
    c->subs_h.resize(P.nsub);
    const int slow = ndim - 1;
    int64_t fac_elems = 0;
    for (int s = 0; s < P.nsub; ++s) {
        int I[3] = {s % P.nb[0], (s / P.nb[0]) % P.nb[1], s / (P.nb[0] * P.nb[1])};
        SubDesc& S = c->subs_h[s];
        std::memset(&S, 0, sizeof(S));
        AxisP axs[3];
        for (int a = 0; a < 3; ++a) {
            S.ib[a] = I[a];
            S.box_lo[a] = blo[a][I[a]];
            S.box_hi[a] = bhi[a][I[a]];
            if (a >= ndim) {
                S.lo[a] = 0;
                S.hi[a] = 1;
                axs[a] = gax[a];
            } else {
                AxisP ax;
                if (I[a] == 0) {
                    ax.lo = 0;
                    ax.left = gax[a].left;
                } else {
                    ax.lo = S.box_lo[a] - P.d - c->W;
                    ax.left = {(double)S.box_lo[a], (double)P.d, (double)c->W};
                }
                if (I[a] == P.nb[a] - 1) {
                    ax.hi = P.N[a];
                    ax.right = gax[a].right;
                } else {
                    ax.hi = S.box_hi[a] + P.d + c->W;
                    ax.right = {(double)S.box_hi[a], (double)P.d, (double)c->W};
                }
                if (ax.lo < 0 || ax.hi > P.N[a])
                    return fail(HELM_ERR_ARG, "subdomain window leaves the grid (boxes too narrow for overlap + sub_pml)");
                S.lo[a] = ax.lo;
                S.hi[a] = ax.hi;
                axs[a] = ax;
            }
            S.nw[a] = S.hi[a] - S.lo[a];
            S.alpha_off[a] = an.size();
            S.face_off[a] = af.size();
            if (a < ndim) {
                fill_window_alpha(axs[a], *pml, omega, an, af);
            } else {
                an.push_back(cd(1, 0));
                af.push_back(cd(1, 0));
                af.push_back(cd(1, 0));
            }
        }
        S.nblk = 1;
        for (int a = 0; a < slow; ++a) S.nblk *= S.nw[a];
        S.nlines = S.nw[slow];
        // padded block size with nbp = 8 (mod 32): the four column planes an
        // m16n8k8 A fragment touches then fall in disjoint shared-memory banks
        {
            const int m16 = (S.nblk + 15) / 16 * 16;
            S.nbp = m16 + ((8 - m16 % 32) + 32) % 32;
        }
        if (S.nbp > 1280) return fail(HELM_ERR_ARG, "subdomain block larger than 1280 nodes");
        S.win_elems = (int64_t)S.nw[0] * S.nw[1] * S.nw[2];
        if (S.win_elems >= ((int64_t)1 << 31)) return fail(HELM_ERR_ARG, "subdomain window of 2^31 nodes or more");
        S.fac_off = fac_elems;
        fac_elems += (int64_t)S.nlines * 2 * S.nbp * S.nbp;
        // couplings between blocks: Pv[p] = prod_{a<slow} alpha_a(node) / h^2,
        // inva[j] = 1 / alpha_slow(face j)
        S.coup_off = pv.size();
        for (int p = 0; p < S.nblk; ++p) {
            cd prod(1.0 / (h * h), 0);
            int rem = p;
            for (int a = 0; a < slow; ++a) {
                int xa = rem % S.nw[a];
                rem /= S.nw[a];
                prod *= an[S.alpha_off[a] + xa];
            }
            pv.push_back(prod);
        }
        S.inva_off = ia.size();
        for (int j = 0; j <= S.nlines; ++j) ia.push_back(1.0 / af[S.face_off[slow] + j]);
        c->nbp_max = std::max(c->nbp_max, S.nbp);
    }
    {
        auto a128 = to_c128(an), f128 = to_c128(af), p128 = to_c128(pv), i128 = to_c128(ia);
        auto a64 = to_c64(an), f64 = to_c64(af), p64 = to_c64(pv), i64 = to_c64(ia);
        TRY(upload(&c->an64, a128.data(), a128.size() * 16, c));
        TRY(upload(&c->af64, f128.data(), f128.size() * 16, c));
        TRY(upload(&c->Pv64, p128.data(), p128.size() * 16, c));
        TRY(upload(&c->inva64, i128.data(), i128.size() * 16, c));
        TRY(upload(&c->an32, a64.data(), a64.size() * 8, c));
        TRY(upload(&c->af32, f64.data(), f64.size() * 8, c));
        TRY(upload(&c->Pv32, p64.data(), p64.size() * 8, c));
        TRY(upload(&c->inva32, i64.data(), i64.size() * 8, c));
        c->inva_count = ia.size();
    }
    {
        std::vector<double> t64(P.d + 1);
        std::vector<float> t32(P.d + 1);
        for (int mm = 0; mm <= P.d; ++mm) {
            t64[mm] = beta_hat((double)mm / P.d);
            t32[mm] = (float)t64[mm];
        }
        TRY(upload(&c->tab64, t64.data(), t64.size() * 8, c));
        TRY(upload(&c->tab32, t32.data(), t32.size() * 4, c));
    }
    TRY(upload(&c->subs_d, c->subs_h.data(), c->subs_h.size() * sizeof(SubDesc), c));
    c->fac_bytes = (size_t)fac_elems * (c->prec == HELM_PREC_F64 ? 8 : 4);

    // ---- routing and dependency levels of one application of Algorithm 3.1/4.1 (or 2.1/2.2)
    auto S = sweep_dirs(ndim, c->cfg.sweep_order);
    auto dirs = transfer_dirs(ndim);
    const int L = c->nsweeps, ns = P.nsub;
    struct Edge {
        int dir[3], sender, l_src;
    };
    std::vector<std::vector<Edge>> inc((size_t)L * ns);
    for (int l = 0; l < L; ++l)
        for (int s = 0; s < ns; ++s) {
            const SubDesc& SD = c->subs_h[s];
            for (auto& d : dirs) {
                int J[3];
                bool ok = true;
                for (int a = 0; a < 3; ++a) {
                    J[a] = SD.ib[a] + d[a];
                    ok &= J[a] >= 0 && J[a] < P.nb[a];
                }
                if (!ok) continue;
                // the receiving sweep: the routing rules (Algorithm 3.1/4.1), or in the
                // additive DDM the step |d|_1 later (Algorithm 2.1/2.2)
                int l2;
                if (c->cfg.algorithm == 1) {
                    l2 = l + std::abs(d[0]) + std::abs(d[1]) + std::abs(d[2]);
                    if (l2 >= L) l2 = -1;
                } else {
                    l2 = route_of(l, d, S, ndim);
                }
                if (l2 < 0) continue;
                int r = J[0] + P.nb[0] * (J[1] + P.nb[1] * J[2]);
                inc[(size_t)l2 * ns + r].push_back({{d[0], d[1], d[2]}, s, l});
            }
        }
    std::vector<char> active((size_t)L * ns, 0);
    for (int s = 0; s < ns; ++s) active[s] = 1;
    for (bool changed = true; changed;) {
        changed = false;
        for (size_t k = 0; k < active.size(); ++k) {
            if (active[k]) continue;
            for (auto& e : inc[k])
                if (active[(size_t)e.l_src * ns + e.sender]) {
                    active[k] = 1;
                    changed = true;
                    break;
                }
        }
    }
    std::vector<int> level((size_t)L * ns, -1);
    std::function<int(size_t)> lev = [&](size_t k) -> int {
        if (level[k] >= 0) return level[k];
        int v = 0;
        for (auto& e : inc[k]) {
            size_t ks = (size_t)e.l_src * ns + e.sender;
            if (active[ks]) v = std::max(v, lev(ks) + 1);
        }
        level[k] = v;
        return v;
    };
    int nlev = 0;
    for (size_t k = 0; k < active.size(); ++k)
        if (active[k]) nlev = std::max(nlev, lev(k) + 1);
    c->node_buf_h.assign((size_t)L * ns, -1);
    int64_t off = 0;
    c->nsolves = 0;
    for (int l = 0; l < L; ++l)
        for (int s = 0; s < ns; ++s) {
            size_t k = (size_t)l * ns + s;
            if (!active[k]) continue;
            c->node_buf_h[k] = off;
            off += c->subs_h[s].win_elems;
            ++c->nsolves;
        }
    c->buf_per_rhs = off;
    std::vector<Incoming> inc_all;
    c->levels.assign(nlev, {});
    for (int l = 0; l < L; ++l)
        for (int s = 0; s < ns; ++s) {
            size_t k = (size_t)l * ns + s;
            if (!active[k]) continue;
            Task t;
            t.sweep = l;
            t.sub = s;
            t.in_off = (int)inc_all.size();
            t.buf_off = c->node_buf_h[k];
            for (auto& e : inc[k]) {
                size_t ks = (size_t)e.l_src * ns + e.sender;
                if (!active[ks]) continue;
                Incoming I;
                for (int a = 0; a < 3; ++a) I.dir[a] = e.dir[a];
                I.sender = e.sender;
                I.sender_buf_off = c->node_buf_h[ks];
                inc_all.push_back(I);
            }
            t.in_cnt = (int)inc_all.size() - t.in_off;
            if (t.in_cnt > 32) return fail(HELM_ERR_ARG, "more than 32 incoming transfers on a subdomain");
            c->levels[level[k]].push_back(t);
        }
    std::vector<Task> all_tasks;
    c->level_off.clear();
    for (auto& lv : c->levels) {
        c->level_off.push_back((int)all_tasks.size());
        all_tasks.insert(all_tasks.end(), lv.begin(), lv.end());
    }
    c->level_off.push_back((int)all_tasks.size());
    TRY(upload(&c->tasks_d, all_tasks.data(), all_tasks.size() * sizeof(Task), c));
    TRY(upload(&c->inc_d, inc_all.data(), inc_all.size() * sizeof(Incoming), c));
    TRY(build_gather_list(c, all_tasks, inc_all));
    TRY(upload(&c->node_buf_d, c->node_buf_h.data(), c->node_buf_h.size() * 8, c));
    CKM(&c->err_d, sizeof(int));
    return HELM_OK;
}

int auto_panel(const helm_ctx* c, int nrhs) {
    int p = c->cfg.rhs_panel;
    if (p <= 0) {
        // measured on GB300 (2D, 184-node lines, 64 RHS): 4 columns per CTA is
        // fastest (panel 8: 2.4x slower, 2: 1.1x, 1: 1.6x)
        p = nrhs >= 16 ? 4 : nrhs >= 2 ? 2 : 1;
    }
    // register budget of solve_kernel: 8 complex64 or 4 complex128 columns per thread
    int pmax = c->prec == HELM_PREC_F64 ? 4 : c->prec == HELM_PREC_TF32 ? 32 : 8;
    if (c->nbp_max > 960) pmax = 2;  // two rows per thread (plane blocks)
    if (p > pmax) p = pmax;
    int q = 1;
    while (q < p) q <<= 1;
    return q;
}

// The subdomain solves of one dependency level (tasks t[0 .. nt)) with the
// kernel the context's precision and factor images select and `panel`
// right-hand sides per CTA where that kernel takes a panel width.
static void launch_level_solve(helm_ctx* c, const Task* t, int nt, int nrhs, int panel) {
    const int64_t rs = c->buf_per_rhs;
    const DevStatus ds{c->err_d, c->wait_polls};
    if (c->prec == HELM_PREC_F64) {
        launch_solve<double>(t, nt, c->subs_d, c->nbp_max, nrhs, panel, static_cast<const double*>(c->fac), c->Pv64,
                             c->inva64, static_cast<cplx<double>*>(c->buf),
                             static_cast<const cplx<double>*>(c->bsrc), rs, ds, c->stream);
        return;
    }
    auto* buf = static_cast<cplx<float>*>(c->buf);
    auto* bsrc = static_cast<const cplx<float>*>(c->bsrc);
    if (c->prec == HELM_PREC_TF32 && c->umma_twist)
        launch_solve_twist(t, nt, c->subs_d, c->umma_nblk, c->umma_lines, nrhs, c->ufac, c->ufac_off, c->ascale_d,
                           c->f16, c->Pv32, c->inva32, buf, bsrc, rs, ds, c->stream);
    else if (c->prec == HELM_PREC_TF32 && c->umma_mt > 0)
        launch_solve_umma(t, nt, c->subs_d, c->umma_nblk, nrhs, panel, static_cast<const float*>(c->ufac),
                          c->ufac_off, c->Pv32, c->inva32, buf, bsrc, rs, ds, c->stream);
    else if (c->prec == HELM_PREC_TF32)
        launch_solve_tc(t, nt, c->subs_d, c->nbp_max, nrhs, panel, static_cast<const float*>(c->fac), c->Pv32,
                        c->inva32, buf, bsrc, rs, ds, c->stream);
    else
        launch_solve<float>(t, nt, c->subs_d, c->nbp_max, nrhs, panel, static_cast<const float*>(c->fac), c->Pv32,
                            c->inva32, buf, bsrc, rs, ds, c->stream);
}

// Autotuner of the right-hand sides per CTA of the subdomain solve.  With
// cfg.rhs_panel set, or for the twisted kernels (panels of 8 fixed by their
// TMEM and register plan), the fixed choice of auto_panel.  Otherwise the
// first batch of each size times every panel width the context's kernel
// takes -- the SIMT kernels 1, 2, 4, 8 (at most 4 in FP64, 2 for plane
// blocks), mma.sync 4, 8, 16, the one-ended tcgen05 kernel 8, 16, 32 -- on
// the widest dependency level, twice each with CUDA events on the context's
// stream (the second run counts), and keeps the fastest for the context's
// lifetime.  A width whose launch the kernel rejects (its shared-memory plan
// does not fit these blocks) is skipped.  The runs only write window buffers,
// which the application then overwrites.
static int tune_panel(helm_ctx* c, int nrhs) {
    const int fixed = auto_panel(c, nrhs);
    if (c->cfg.rhs_panel > 0 || (c->prec == HELM_PREC_TF32 && c->umma_twist) || c->levels.empty()) return fixed;
    auto it = c->panel_pick.find(nrhs);
    if (it != c->panel_pick.end()) return it->second;
    std::vector<int> cand;
    if (c->prec == HELM_PREC_TF32 && c->umma_mt > 0)
        cand = {8, 16, 32};
    else if (c->prec == HELM_PREC_TF32)
        cand = {4, 8, 16};
    else {
        const int pmax = c->nbp_max > 960 ? 2 : c->prec == HELM_PREC_F64 ? 4 : 8;
        for (int p = 1; p <= pmax; p *= 2) cand.push_back(p);
    }
    size_t widest = 0;
    for (size_t lv = 1; lv < c->levels.size(); ++lv)
        if (c->levels[lv].size() > c->levels[widest].size()) widest = lv;
    const Task* t = c->tasks_d + c->level_off[widest];
    const int nt = (int)c->levels[widest].size();
    if (cudaPeekAtLastError() != cudaSuccess) return fixed;  // leave an earlier error to its reporter
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fixed;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fixed;
    }
    int best = fixed;
    float best_ms = -1.f;
    for (int p : cand) {
        float ms = 0.f;
        bool launched = true;
        for (int rep = 0; rep < 2 && launched; ++rep) {
            cudaEventRecord(e0, c->stream);
            launch_level_solve(c, t, nt, nrhs, p);
            launched = cudaGetLastError() == cudaSuccess;
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (launched && (best_ms < 0.f || ms < best_ms)) best = p, best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->panel_pick[nrhs] = best;
    return best;
}

// One application of Algorithm 3.1 / 4.1 to the J-scaled source b (device,
// [nrhs][grid], complex128 or float-float); the assembled u_DDM goes to U
// (device, the same form).
template <typename VB>
int apply_ddm_dev(helm_ctx* c, int nrhs, const VB* b, VB* U) {
    if (!c->factored) return fail(HELM_ERR_NOT_FACTORED, "call helm_factor first");
    TRY(ensure_buffers(c, nrhs));
    const int64_t rs = c->buf_per_rhs;
    const int panel = tune_panel(c, nrhs);
    const double es = (double)elem_size(c);
    for (size_t lv = 0; lv < c->levels.size(); ++lv) {
        const Task* t = c->tasks_d + c->level_off[lv];
        int nt = (int)c->levels[lv].size();
        // gather: the work list's sources written (the reads depend on the strips)
        const double gbytes = (double)c->gnodes_lv[lv] * nrhs * es;
        double sbytes = 0, sflops = 0;
        for (const Task& tk : c->levels[lv]) {
            const SubDesc& S = c->subs_h[tk.sub];
            const double n = S.nblk, nl = S.nlines, passes = 2.0 * nl - 1.0;
            // block inverses once per pass, counted at the factors' complex storage size
            // (8 bytes per entry for complex64, 16 for complex128) whatever image the kernel
            // streams (the FP16 tensor-core image holds 4 bytes per entry), + b in, y out, y in,
            // u out
            sbytes += passes * n * n * es + 4.0 * nl * n * nrhs * es;
            sflops += passes * n * n * nrhs * 8.0;
        }
        if (c->prec == HELM_PREC_F64) {
            auto* buf = static_cast<cplx<double>*>(c->buf);
            auto* bsrc = static_cast<cplx<double>*>(c->bsrc);
            {
                ProfScope ps(c, HELM_K_GATHER, 1, gbytes);
                launch_gather<double>(c->gblk_d + c->gblk_off[lv], c->gblk_off[lv + 1] - c->gblk_off[lv],
                                      c->gnode_d, c->tasks_d, c->subs_d, c->inc_d, c->P, c->m64, c->an64,
                                      c->af64, c->tab64, b, nrhs, buf, bsrc, rs, c->stream);
            }
            ProfScope ps(c, HELM_K_SOLVE, 1, sbytes, sflops);
            launch_level_solve(c, t, nt, nrhs, panel);
        } else {
            auto* buf = static_cast<cplx<float>*>(c->buf);
            auto* bsrc = static_cast<cplx<float>*>(c->bsrc);
            {
                ProfScope ps(c, HELM_K_GATHER, 1, gbytes);
                launch_gather<float>(c->gblk_d + c->gblk_off[lv], c->gblk_off[lv + 1] - c->gblk_off[lv],
                                     c->gnode_d, c->tasks_d, c->subs_d, c->inc_d, c->P, c->m32, c->an32,
                                     c->af32, c->tab32, b, nrhs, buf, bsrc, rs, c->stream);
            }
            ProfScope ps(c, HELM_K_SOLVE, 1, sbytes, sflops);
            launch_level_solve(c, t, nt, nrhs, panel);
        }
    }
    ProfScope ps(c, HELM_K_ASSEMBLE, 1, (double)c->Ng * nrhs * 16.0);
    if (c->prec == HELM_PREC_F64)
        launch_assemble<double>(c->P, c->subs_d, c->box_of, c->node_buf_d, c->nsweeps, c->tab64,
                                static_cast<const cplx<double>*>(c->buf), rs, nrhs, U, c->stream);
    else
        launch_assemble<float>(c->P, c->subs_d, c->box_of, c->node_buf_d, c->nsweeps, c->tab32,
                               static_cast<const cplx<float>*>(c->buf), rs, nrhs, U, c->stream);
    CK(cudaGetLastError());
    return HELM_OK;
}

// ---- host <-> device staging of caller data: a caller's host array goes
// through one of the context's staging buffers (slot 0, 1, 2 in the order of a
// call's arguments), kept between calls so that no call allocates or frees
// device memory once they have grown; a device array is used in place.
struct Staged {
    cplx<double>* ptr = nullptr;
};

int stage_in(helm_ctx* c, const void* src, size_t bytes, int mem, Staged& out, int slot) {
    if (mem == HELM_MEM_DEVICE) {
        out.ptr = (cplx<double>*)src;
        return HELM_OK;
    }
    if (mem != HELM_MEM_HOST) return fail(HELM_ERR_ARG, "mem must be HELM_MEM_HOST or HELM_MEM_DEVICE");
    if (bytes > c->stage_cap[slot]) {
        if (c->stage_d[slot]) {
            CK(cudaFree(c->stage_d[slot]));
            c->dev_bytes -= c->stage_cap[slot];
        }
        c->stage_d[slot] = nullptr;
        c->stage_cap[slot] = 0;
        CKM(&c->stage_d[slot], bytes);
        c->stage_cap[slot] = bytes;
        c->dev_bytes += bytes;
    }
    out.ptr = c->stage_d[slot];
    if (src) CK(cudaMemcpyAsync(out.ptr, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return HELM_OK;
}

// Device error word of the context: 1 = bad pivot in a factor, 2 = a bounded
// wait in a kernel expired.  Read (and cleared) at the end of every call.
int check_device_error(helm_ctx* c) {
    int err = 0;
    CK(cudaMemcpyAsync(&err, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (err == 0) return HELM_OK;
    CK(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (err == 2) return fail(HELM_ERR_TIMEOUT, "a bounded device wait expired");
    return fail(HELM_ERR_NUMERIC, "numerical breakdown flagged on the device");
}

int stage_out(helm_ctx* c, void* dst, const Staged& s, size_t bytes, int mem) {
    if (mem == HELM_MEM_HOST) CK(cudaMemcpyAsync(dst, s.ptr, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    resolve_profile(c);
    return check_device_error(c);
}

int ensure_gm(helm_ctx* c, int nrhs, int count) {
    if (nrhs > c->gm_rhs) {
        for (auto* p : c->gm) cudaFree(p);
        c->dev_bytes -= c->gm.size() * (size_t)c->gm_rhs * c->Ng * 16;
        c->gm.clear();
        c->gm_rhs = nrhs;
    }
    while ((int)c->gm.size() < count) {
        cplx<double>* p = nullptr;
        CKM(&p, (size_t)c->gm_rhs * c->Ng * 16);
        c->dev_bytes += (size_t)c->gm_rhs * c->Ng * 16;
        c->gm.push_back(p);
    }
    return HELM_OK;
}

// FP64 flexible GMRES, right preconditioned by one DDM application per
// iteration (Remark 1), on A u = b with b on the device.  Restarts every
// cfg.restart iterations; stops when every RHS has |b - A u| <= rtol |b|.
int gmres_dev(helm_ctx* c, int nrhs, const cplx<double>* b, cplx<double>* x, double rtol,
              int maxit, helm_stats* st, int restart) {
    const int m = restart;
    const int64_t Ng = c->Ng;
    // vectors, allocated as the Krylov space grows: scratch w (0), then
    // V_i at 1 + 2i and Z_i at 2 + 2i
    TRY(ensure_gm(c, nrhs, 2));
    TRY(ensure_small(c, (size_t)2 * (m + 2) * nrhs));  // coefficients, then the fused kernels' dots
    const int nblk = (int)std::min<int64_t>(256, (Ng + 4095) / 4096);
    // work vectors in float-float form (one float4 per complex entry)
    auto fv = [&](int i) { return reinterpret_cast<float4*>(c->gm[i]); };
    float4* w = fv(0);
    auto V = [&](int i) { return fv(1 + 2 * i); };
    auto Z = [&](int i) { return fv(2 + 2 * i); };
    std::vector<double> bn(nrhs), res(nrhs, 1.0);
    std::vector<cplx<double>> hd((size_t)(m + 2) * nrhs);
    auto norms = [&](const auto* v, std::vector<double>& out) -> int {
        { ProfScope ps_(c, HELM_K_KRYLOV, 2); launch_norms2(v, Ng, nrhs, c->small_d, c->partial_d, nblk, c->stream); }
        CK(cudaMemcpyAsync(hd.data(), c->small_d, nrhs * 16, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int r = 0; r < nrhs; ++r) out[r] = std::sqrt(std::max(0.0, hd[r].re));
        return HELM_OK;
    };
    CK(cudaMemsetAsync(x, 0, (size_t)nrhs * Ng * 16, c->stream));
    TRY(norms(b, bn));
    for (auto& v : bn)
        if (v == 0) v = 1;
    int total = 0, apps = 0;
    double maxres = 0;
    bool conv = false;
    for (bool first = true;; first = false) {
        // r = b - A x: b itself while x is still zero
        if (first) {
            ProfScope ps_(c, HELM_K_KRYLOV, 1);
            launch_to_ff(b, w, (int64_t)nrhs * Ng, c->stream);
        } else {
            // x in float-float form first (into u_0's buffer, free until the swap
            // below): the operator product then reads no FP64 neighbours
            ProfScope ps_(c, HELM_K_KRYLOV, 2);
            launch_to_ff(x, fv(1), (int64_t)nrhs * Ng, c->stream);
            launch_apply_A(c->P, c->stc_d, b, static_cast<const float4*>(fv(1)), w, nrhs, c->stream);
        }
        std::vector<double> beta(nrhs);
        TRY(norms(w, beta));
        maxres = 0;
        for (int r = 0; r < nrhs; ++r) {
            res[r] = beta[r] / bn[r];
            maxres = std::max(maxres, res[r]);
        }
        if (c->cfg.verbose) fprintf(stderr, "[helm] gmres it %d max rel resid %.3e\n", total, maxres);
        if (maxres <= rtol) {
            conv = true;
            break;
        }
        if (total >= maxit) break;
        // The basis is kept unnormalised: u_i = s_i v_i with the scale s_i of
        // every right-hand side held here, folded into the Gram-Schmidt
        // coefficients (u_i^H w = s_i v_i^H w; w - sum (v_i^H w) v_i =
        // w - sum (u_i^H w / s_i^2) u_i) and the final combination
        // (z'_k = M^-1 u_k = s_k z_k).  u_0 = r_0 is w itself: the buffers swap.
        std::swap(c->gm[0], c->gm[1]);
        w = fv(0);
        std::vector<std::vector<double>> sv(m + 1, std::vector<double>(nrhs, 1.0));
        for (int r = 0; r < nrhs; ++r) sv[0][r] = beta[r] > 0 ? beta[r] : 1.0;
        // per-RHS Hessenberg (column-major, (m+1) x m), Givens, residual vector g
        std::vector<std::vector<cd>> H(nrhs, std::vector<cd>((size_t)(m + 1) * m, 0.0));
        std::vector<std::vector<double>> cs(nrhs, std::vector<double>(m, 0));
        std::vector<std::vector<cd>> sn(nrhs, std::vector<cd>(m, 0.0));
        std::vector<std::vector<cd>> g(nrhs, std::vector<cd>(m + 1, 0.0));
        std::vector<int> kc(nrhs, 0);
        std::vector<char> done(nrhs, 0);
        for (int r = 0; r < nrhs; ++r) {
            g[r][0] = beta[r];
            if (res[r] <= rtol) done[r] = 1;
        }
        int k = 0;
        for (; k < m && total < maxit; ++k) {
            TRY(ensure_gm(c, nrhs, 2 * k + 4));  // Z_k and V_{k+1}
            w = fv(0);
            TRY(apply_ddm_dev(c, nrhs, V(k), Z(k)));
            ++apps;
            // w = -A z'_k (apply_A with no b); CGS2 on w against the u_i: the
            // dots d = U^H w, then w -= sum (d_i / s_i^2) u_i, twice.  The
            // first combination also forms the second pass's dots, the second
            // the norm of what is left (fused kernels when k + 1 <= 8).  With
            // h_i = sum over the passes of d_i / s_i (= v_i^H w):
            //   A z_k = sum_i (-h_i / s_k) v_i - (|w| / s_k) v_{k+1},
            // v_{k+1} = w / |w|, stored unnormalised as u_{k+1} = w, s_{k+1} = |w|.
            {
                ProfScope ps_(c, HELM_K_KRYLOV, 1);
                launch_apply_A(c->P, c->stc_d, nullptr, Z(k), w, nrhs, c->stream);
            }
            std::vector<std::vector<cd>> hsum(nrhs, std::vector<cd>(k + 2, 0.0));
            {
                std::vector<float4*> vp(k + 1);
                for (int i = 0; i <= k; ++i) vp[i] = V(i);
                CK(cudaMemcpyAsync(c->vptr_d, vp.data(), vp.size() * sizeof(void*),
                                   cudaMemcpyHostToDevice, c->stream));
            }
            const bool fused = k + 1 <= kComboDotsMax;
            std::vector<cplx<double>> coef((size_t)(k + 1) * nrhs);
            // dots d (in hd) -> h sums and the combination coefficients -d_i / s_i^2
            auto take_dots = [&]() {
                for (int i = 0; i <= k; ++i)
                    for (int r = 0; r < nrhs; ++r) {
                        const cd d(hd[(size_t)i * nrhs + r].re, hd[(size_t)i * nrhs + r].im);
                        hsum[r][i] += d / sv[i][r];
                        const cd cf = -d / (sv[i][r] * sv[i][r]);
                        coef[(size_t)i * nrhs + r] = {cf.real(), cf.imag()};
                    }
                return cudaMemcpyAsync(c->small_d, coef.data(), coef.size() * 16, cudaMemcpyHostToDevice,
                                       c->stream);
            };
            auto fetch = [&](size_t count) -> int {
                CK(cudaMemcpyAsync(hd.data(), c->small_d, count * 16, cudaMemcpyDeviceToHost, c->stream));
                CK(cudaStreamSynchronize(c->stream));
                return HELM_OK;
            };
            {
                ProfScope ps_(c, HELM_K_KRYLOV, mdots_launches(k + 1));
                launch_mdots(c->vptr_d, k + 1, w, Ng, nrhs, c->small_d, c->partial_d, nblk, c->stream);
            }
            TRY(fetch((size_t)(k + 1) * nrhs));
            CK(take_dots());
            std::vector<double> wn(nrhs);
            if (fused) {
                {
                    ProfScope ps_(c, HELM_K_KRYLOV, 2);
                    CK(launch_combo_dots(w, c->vptr_d, k + 1, c->small_d, Ng, nrhs, true,
                                         c->small_d + coef.size(), c->partial_d, nblk, c->stream));
                }
                CK(cudaMemcpyAsync(hd.data(), c->small_d + coef.size(), coef.size() * 16, cudaMemcpyDeviceToHost,
                                   c->stream));
                CK(cudaStreamSynchronize(c->stream));
                CK(take_dots());
                {
                    ProfScope ps_(c, HELM_K_KRYLOV, 2);
                    CK(launch_combo_dots(w, c->vptr_d, k + 1, c->small_d, Ng, nrhs, false,
                                         c->small_d + coef.size(), c->partial_d, nblk, c->stream));
                }
                CK(cudaMemcpyAsync(hd.data(), c->small_d + coef.size(), nrhs * 16, cudaMemcpyDeviceToHost,
                                   c->stream));
                CK(cudaStreamSynchronize(c->stream));
                for (int r = 0; r < nrhs; ++r) wn[r] = std::sqrt(std::max(0.0, hd[r].re));
            } else {
                { ProfScope ps_(c, HELM_K_KRYLOV, 1); launch_mcombo(w, c->vptr_d, k + 1, c->small_d, Ng, nrhs, 1.0, c->stream); }
                {
                    ProfScope ps_(c, HELM_K_KRYLOV, mdots_launches(k + 1));
                    launch_mdots(c->vptr_d, k + 1, w, Ng, nrhs, c->small_d + coef.size(), c->partial_d, nblk,
                                 c->stream);
                }
                CK(cudaMemcpyAsync(hd.data(), c->small_d + coef.size(), coef.size() * 16, cudaMemcpyDeviceToHost,
                                   c->stream));
                CK(cudaStreamSynchronize(c->stream));
                CK(take_dots());
                { ProfScope ps_(c, HELM_K_KRYLOV, 1); launch_mcombo(w, c->vptr_d, k + 1, c->small_d, Ng, nrhs, 1.0, c->stream); }
                TRY(norms(w, wn));
            }
            TRY(check_device_error(c));  // a timed-out preconditioner ends the solve here
            // u_{k+1} = w: the buffers swap
            std::swap(c->gm[0], c->gm[1 + 2 * (k + 1)]);
            w = fv(0);
            for (int r = 0; r < nrhs; ++r) sv[k + 1][r] = wn[r] > 1e-300 ? wn[r] : 1.0;
            ++total;
            bool all = true;
            maxres = 0;
            for (int r = 0; r < nrhs; ++r) {
                if (done[r]) continue;
                std::vector<cd>& Hr = H[r];
                for (int i = 0; i <= k; ++i) Hr[(size_t)k * (m + 1) + i] = -hsum[r][i] / sv[k][r];
                Hr[(size_t)k * (m + 1) + k + 1] = -wn[r] / sv[k][r];
                for (int i = 0; i < k; ++i) {
                    cd a = Hr[(size_t)k * (m + 1) + i], bb = Hr[(size_t)k * (m + 1) + i + 1];
                    Hr[(size_t)k * (m + 1) + i] = cs[r][i] * a + sn[r][i] * bb;
                    Hr[(size_t)k * (m + 1) + i + 1] = -std::conj(sn[r][i]) * a + cs[r][i] * bb;
                }
                cd a = Hr[(size_t)k * (m + 1) + k], bb = Hr[(size_t)k * (m + 1) + k + 1];
                double t = std::sqrt(std::norm(a) + std::norm(bb));
                if (std::abs(a) == 0) {
                    cs[r][k] = 0;
                    sn[r][k] = 1;
                    Hr[(size_t)k * (m + 1) + k] = bb;
                } else {
                    cs[r][k] = std::abs(a) / t;
                    sn[r][k] = (a / std::abs(a)) * std::conj(bb) / t;
                    Hr[(size_t)k * (m + 1) + k] = (a / std::abs(a)) * t;
                }
                Hr[(size_t)k * (m + 1) + k + 1] = 0;
                g[r][k + 1] = -std::conj(sn[r][k]) * g[r][k];
                g[r][k] = cs[r][k] * g[r][k];
                kc[r] = k + 1;
                double est = std::abs(g[r][k + 1]) / bn[r];
                res[r] = est;
                if (est <= rtol) done[r] = 1;
                maxres = std::max(maxres, est);
                all = all && done[r];
            }
            if (c->cfg.verbose) fprintf(stderr, "[helm]   inner %d est %.3e\n", total, maxres);
            if (all) {
                ++k;
                break;
            }
        }
        // y = R^{-1} g per RHS, then x += sum_i y_i Z_i
        std::vector<cplx<double>> coef((size_t)k * nrhs, {0, 0});
        for (int r = 0; r < nrhs; ++r) {
            int kk = kc[r];
            std::vector<cd> y(kk, 0.0);
            for (int i = kk - 1; i >= 0; --i) {
                cd s = g[r][i];
                for (int j2 = i + 1; j2 < kk; ++j2) s -= H[r][(size_t)j2 * (m + 1) + i] * y[j2];
                y[i] = s / H[r][(size_t)i * (m + 1) + i];
            }
            // x += sum y_i z_i = sum (y_i / s_i) z'_i
            for (int i = 0; i < kk; ++i) coef[(size_t)i * nrhs + r] = {y[i].real() / sv[i][r], y[i].imag() / sv[i][r]};
        }
        CK(cudaMemcpyAsync(c->small_d, coef.data(), coef.size() * 16, cudaMemcpyHostToDevice,
                           c->stream));
        if (k > 0) {
            std::vector<float4*> zp(k);
            for (int i = 0; i < k; ++i) zp[i] = Z(i);
            CK(cudaMemcpyAsync(c->zptr_d, zp.data(), zp.size() * sizeof(void*),
                               cudaMemcpyHostToDevice, c->stream));
            { ProfScope ps_(c, HELM_K_KRYLOV, 1); launch_mcombo(x, c->zptr_d, k, c->small_d, Ng, nrhs, 1.0, c->stream); }
        }
        CK(cudaStreamSynchronize(c->stream));
    }
    if (st) {
        st->iters = total;
        st->applications = apps;
        st->resid = maxres;
        st->levels = (int)c->levels.size();
        st->solves = c->nsolves;
    }
    CK(cudaGetLastError());
    if (!conv) return fail(HELM_ERR_NO_CONVERGENCE, "GMRES reached maxit");
    return HELM_OK;
}

// The DDM as a stationary iteration (Section 5.2.2): u_0 = 0,
// u_{k+1} = u_k + M (b - A u_k).  The residual goes to work vector 0 and the
// correction M r to work vector 1 (float-float); the solution is updated by
// the combination kernel with coefficient 1.
int stationary_dev(helm_ctx* c, int nrhs, const cplx<double>* b, cplx<double>* x, double rtol, int maxit,
                   helm_stats* st) {
    const int64_t Ng = c->Ng;
    TRY(ensure_gm(c, nrhs, 2));
    TRY(ensure_small(c, (size_t)2 * nrhs));
    const int nblk = (int)std::min<int64_t>(256, (Ng + 4095) / 4096);
    std::vector<cplx<double>> hd(nrhs);
    auto norms = [&](const auto* v, std::vector<double>& out) -> int {
        { ProfScope ps_(c, HELM_K_KRYLOV, 2); launch_norms2(v, Ng, nrhs, c->small_d, c->partial_d, nblk, c->stream); }
        CK(cudaMemcpyAsync(hd.data(), c->small_d, nrhs * 16, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int r = 0; r < nrhs; ++r) out[r] = std::sqrt(std::max(0.0, hd[r].re));
        return HELM_OK;
    };
    CK(cudaMemsetAsync(x, 0, (size_t)nrhs * Ng * 16, c->stream));
    std::vector<double> bn(nrhs), rn(nrhs);
    TRY(norms(b, bn));
    for (auto& v : bn)
        if (v == 0) v = 1;
    const std::vector<cplx<double>> one(nrhs, cplx<double>{1.0, 0.0});
    int apps = 0;
    double maxres = 0;
    bool conv = false;
    while (true) {
        float4* r = reinterpret_cast<float4*>(c->gm[0]);
        float4* z = reinterpret_cast<float4*>(c->gm[1]);
        { ProfScope ps_(c, HELM_K_KRYLOV, 1); launch_apply_A(c->P, c->stc_d, b, x, r, nrhs, c->stream); }
        TRY(norms(r, rn));
        maxres = 0;
        for (int q = 0; q < nrhs; ++q) maxres = std::max(maxres, rn[q] / bn[q]);
        if (c->cfg.verbose) fprintf(stderr, "[helm] iteration %d max rel resid %.3e\n", apps, maxres);
        if (maxres <= rtol) {
            conv = true;
            break;
        }
        if (apps >= maxit) break;
        TRY(apply_ddm_dev(c, nrhs, static_cast<const float4*>(r), z));
        ++apps;
        TRY(check_device_error(c));  // a timed-out subdomain solve ends the iteration here
        CK(cudaMemcpyAsync(c->small_d, one.data(), nrhs * 16, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->zptr_d, &z, sizeof(float4*), cudaMemcpyHostToDevice, c->stream));
        { ProfScope ps_(c, HELM_K_KRYLOV, 1); launch_mcombo(x, c->zptr_d, 1, c->small_d, Ng, nrhs, 1.0, c->stream); }
    }
    if (st) {
        st->iters = apps;
        st->applications = apps;
        st->resid = maxres;
        st->levels = (int)c->levels.size();
        st->solves = c->nsolves;
    }
    CK(cudaGetLastError());
    if (!conv) return fail(HELM_ERR_NO_CONVERGENCE, "the stationary iteration reached maxit");
    return HELM_OK;
}

// The subdomain solve of one task (device descriptor `task`, sweep 0) in place
// on the window buffer wb ([nrhs][window] in the working precision, local
// sources and solution in the same array), with the kernel the context's
// precision selects -- the same choice the DDM application makes.  Queued on
// the context's stream; allocates nothing.
void launch_one_subdomain_solve(helm_ctx* c, const Task* task, int nrhs, void* wb, int64_t we) {
    const int panel = auto_panel(c, nrhs);
    const DevStatus ds{c->err_d, c->wait_polls};
    if (c->prec == HELM_PREC_F64) {
        auto* b = static_cast<cplx<double>*>(wb);
        launch_solve<double>(task, 1, c->subs_d, c->nbp_max, nrhs, panel, static_cast<const double*>(c->fac),
                             c->Pv64, c->inva64, b, b, we, ds, c->stream);
        return;
    }
    auto* b = static_cast<cplx<float>*>(wb);
    if (c->prec == HELM_PREC_TF32 && c->umma_twist)
        launch_solve_twist(task, 1, c->subs_d, c->umma_nblk, c->umma_lines, nrhs, c->ufac, c->ufac_off, c->ascale_d,
                           c->f16, c->Pv32, c->inva32, b, b, we, ds, c->stream);
    else if (c->prec == HELM_PREC_TF32 && c->umma_mt > 0)
        launch_solve_umma(task, 1, c->subs_d, c->umma_nblk, nrhs, panel, static_cast<const float*>(c->ufac),
                          c->ufac_off, c->Pv32, c->inva32, b, b, we, ds, c->stream);
    else if (c->prec == HELM_PREC_TF32)
        launch_solve_tc(task, 1, c->subs_d, c->nbp_max, nrhs, panel, static_cast<const float*>(c->fac), c->Pv32,
                        c->inva32, b, b, we, ds, c->stream);
    else
        launch_solve<float>(task, 1, c->subs_d, c->nbp_max, nrhs, panel, static_cast<const float*>(c->fac),
                            c->Pv32, c->inva32, b, b, we, ds, c->stream);
}

void noalloc_solve_cb(void* ctx, const Task* task, int nrhs, void* wb, int64_t we) {
    launch_one_subdomain_solve(static_cast<helm_ctx*>(ctx), task, nrhs, wb, we);
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

// ============================================================================= C ABI
extern "C" {

int helm_setup(helm_ctx** out, int ndim, const int64_t n[3], double h, double omega,
               const double* m, const helm_pml* pml, const helm_partition* part,
               const helm_config* cfg) {
    if (!out) return fail(HELM_ERR_ARG, "out is null");
    *out = nullptr;
    helm_ctx* c = new helm_ctx();
    int rc = setup_impl(c, ndim, n, h, omega, m, pml, part, cfg);
    if (rc != HELM_OK) {
        std::string keep = g_last_error;
        helm_destroy(c);
        g_last_error = keep;
        return rc;
    }
    *out = c;
    return HELM_OK;
}

int helm_factor(helm_ctx* c) {
    if (!c) return fail(HELM_ERR_ARG, "null context");
    if (c->factored) return HELM_OK;
    double t0 = now_ms();
    c->panel_pick.clear();
    if (!c->fac) {
        CKM(&c->fac, c->fac_bytes);
        c->dev_bytes += c->fac_bytes;
    }
    CK(cudaMemsetAsync(c->fac, 0, c->fac_bytes, c->stream));
    CK(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->stream));
    double fbytes = 0, fflops = 0;
    for (const SubDesc& S : c->subs_h) {
        fbytes += (double)S.nlines * S.nblk * S.nblk * elem_size(c);
        fflops += (double)S.nlines * 8.0 * S.nblk * S.nblk * S.nblk;
    }
    ProfScope ps_(c, HELM_K_FACTOR, 1, fbytes, fflops);
    if (c->prec == HELM_PREC_F64)
        launch_factor_f64(c->subs_d, c->P.nsub, c->nbp_max, c->P, c->m64, c->an64, c->af64,
                          static_cast<double*>(c->fac), c->err_d, c->stream);
    else
        launch_factor_f32(c->subs_d, c->P.nsub, c->nbp_max, c->P, c->m32, c->an32, c->af32,
                          static_cast<float*>(c->fac), c->err_d, c->stream);
    if (c->prec == HELM_PREC_TF32) {
        int nblk_max = 0, nl_min = 1 << 30, nl_max = 0;
        for (const SubDesc& S : c->subs_h) {
            nblk_max = std::max(nblk_max, S.nblk);
            nl_min = std::min(nl_min, S.nlines);
            nl_max = std::max(nl_max, S.nlines);
        }
        // default: the twisted kernel (2 tiles, or 3 with FP16 operands), else the one-ended one
        const int tk = c->cfg.tc_kernel;
        const bool twist = tk == 0 && twist_supported(nblk_max, nl_min, nl_max, c->f16);
        const bool umma = tk != 1 && (twist || umma_supported(nblk_max));
        float* fac2 = nullptr;
        if (twist) {
            // the far half of every subdomain's lines, eliminated from the far end
            // (before the standard factors are rounded: the middle block uses one)
            CKM(&fac2, c->fac_bytes);
            launch_factor_twist_f32(c->subs_d, c->P.nsub, c->nbp_max, c->P, c->m32, c->an32, c->af32,
                                    static_cast<const float*>(c->fac), fac2, c->err_d, c->stream);
        }
        launch_round_tf32(static_cast<float*>(c->fac), (int64_t)(c->fac_bytes / sizeof(float)),
                          c->stream);
        if (umma) {
            c->umma_twist = twist;
            c->umma_mt = twist ? 1 : umma_tiles(nblk_max);
            c->umma_nblk = nblk_max;
            c->umma_lines = nl_max;
            const bool f16 = twist && c->f16;
            std::vector<int64_t> off;
            int64_t tot = 0;
            int max_lines = 0;
            for (const SubDesc& S : c->subs_h) {
                off.push_back(tot);
                tot += f16 ? twist_f16_factor_bytes(S) : umma_factor_bytes(S, c->umma_mt);
                max_lines = std::max(max_lines, S.nlines);
            }
            if (!c->ufac) {
                CKM(&c->ufac, (size_t)tot);
                c->dev_bytes += (size_t)tot;
                c->ufac_bytes = (size_t)tot;
                TRY(upload(&c->ufac_off, off.data(), off.size() * sizeof(int64_t), c));
            }
            if (f16) {
                if (!c->ascale_d) {
                    CKM(&c->ascale_d, c->inva_count * sizeof(int));
                    c->dev_bytes += c->inva_count * sizeof(int);
                }
                launch_line_scales(c->subs_d, c->P.nsub, max_lines, static_cast<const float*>(c->fac), fac2,
                                   c->ascale_d, c->stream);
                launch_repack_f16(c->subs_d, c->subs_h, static_cast<const float*>(c->fac), fac2, c->ascale_d,
                                  c->ufac_off, c->ufac, c->stream);
            } else {
                launch_repack_umma(c->subs_d, c->subs_h, c->umma_mt, static_cast<const float*>(c->fac), fac2,
                                   c->ufac_off, static_cast<float*>(c->ufac), c->stream);
            }
        }
        if (fac2) {
            CK(cudaStreamSynchronize(c->stream));
            CK(cudaFree(fac2));
        }
    }
    CK(cudaGetLastError());
    int err = 0;
    CK(cudaMemcpyAsync(&err, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (err) return fail(HELM_ERR_NUMERIC, "zero or non-finite pivot in a subdomain factor");
    c->factored = true;
    c->t_factor_ms = now_ms() - t0;
    return HELM_OK;
}

int helm_apply_ddm(helm_ctx* c, int nrhs, const void* F, void* U, int mem) {
    if (!c || !F || !U || nrhs < 1) return fail(HELM_ERR_ARG, "bad argument");
    if (!c->factored) return fail(HELM_ERR_NOT_FACTORED, "call helm_factor first");
    size_t bytes = (size_t)nrhs * c->Ng * 16;
    Staged f, u;
    TRY(stage_in(c, F, bytes, mem, f, 0));
    TRY(stage_in(c, mem == HELM_MEM_DEVICE ? U : nullptr, bytes, mem, u, 1));
    TRY(ensure_bvec(c, nrhs));
    { ProfScope ps_(c, HELM_K_KRYLOV, 1); launch_scale_J(c->P, c->gwin, f.ptr, c->bvec, nrhs, false, c->stream); }
    TRY(apply_ddm_dev(c, nrhs, c->bvec, u.ptr));
    return stage_out(c, U, u, bytes, mem);
}

// Right-hand sides per GMRES run and the restart length, so that the run's
// device memory fits: its window buffers (local sources and solutions of every
// subdomain solve) and its Krylov vectors (2 restart + 2 float-float vectors),
// against the free device memory plus what the
// context already holds in those buffers (and cfg.max_device_bytes, when set).
// The whole batch when it fits with the configured restart; else the largest
// halving of it that fits with a restart of at least 8 (the restart lowered to
// what fits); else halving on with a restart of 8.
void solve_plan(const helm_ctx* c, int nrhs, int maxit, bool gmres, int* chunk, int* restart) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    size_t held = 2 * (size_t)c->cap_rhs * c->buf_per_rhs * elem_size(c);
    held += c->gm.size() * (size_t)c->gm_rhs * c->Ng * 16;
    const size_t reserve = (size_t)1 << 30;
    double avail = (double)free_b + (double)held - (double)reserve;
    if (c->cfg.max_device_bytes > 0)
        avail = std::min(avail, (double)c->cfg.max_device_bytes - (double)(c->dev_bytes - held));
    const int mcfg = std::max(1, std::min(c->cfg.restart, maxit));
    const int mmin = std::min(8, mcfg);
    auto per_rhs = [&](int m) {
        const double vecs = gmres ? 2.0 * m + 2.0 : 2.0;
        return 2.0 * c->buf_per_rhs * elem_size(c) + vecs * c->Ng * 16.0;
    };
    int C = nrhs;
    if (C * per_rhs(mcfg) > avail) {
        while (C > 1 && C * per_rhs(mmin) > avail) C = (C + 1) / 2;
    }
    int m = mcfg;
    while (m > mmin && C * per_rhs(m) > avail) --m;
    *chunk = C;
    *restart = m;
}

// Copies of a chunked solve with host buffers: every chunk's input goes on
// the context's copy stream up front (event `in`), each chunk's output after
// its solve (event `out` on the compute stream), so that chunk k+1's upload
// and chunk k-1's download overlap chunk k's solve.  The destructor waits for
// the copy stream (no copy touches the caller's buffers after the call) and
// frees the events.
struct ChunkCopies {
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> in, out;
    ~ChunkCopies() {
        if (cs) cudaStreamSynchronize(cs);
        for (auto e : in) cudaEventDestroy(e);
        for (auto e : out) cudaEventDestroy(e);
    }
};

static int solve_common(helm_ctx* c, int nrhs, const void* F, void* U, int mem, double rtol,
                        int maxit, helm_stats* st, bool adjoint, bool stationary = false) {
    if (!c || !F || !U || nrhs < 1 || !(rtol > 0) || maxit < 1)
        return fail(HELM_ERR_ARG, "bad argument");
    if (!c->factored) return fail(HELM_ERR_NOT_FACTORED, "call helm_factor first");
    if (mem != HELM_MEM_HOST && mem != HELM_MEM_DEVICE)
        return fail(HELM_ERR_ARG, "mem must be HELM_MEM_HOST or HELM_MEM_DEVICE");
    double t0 = now_ms();
    const bool host = mem == HELM_MEM_HOST;
    size_t bytes = (size_t)nrhs * c->Ng * 16;
    Staged f, u;
    // host buffers: device staging only here, the copies go chunk by chunk below
    TRY(stage_in(c, host ? nullptr : F, bytes, mem, f, 0));
    TRY(stage_in(c, host ? nullptr : U, bytes, mem, u, 1));
    TRY(ensure_bvec(c, nrhs));
    int chunk = nrhs, restart = c->cfg.restart;
    solve_plan(c, nrhs, maxit, !stationary, &chunk, &restart);
    const int nchunk = (nrhs + chunk - 1) / chunk;
    ChunkCopies cc;
    if (host) {
        if (!c->cstream) CK(cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
        cc.cs = c->cstream;
        for (int k = 0; k < nchunk; ++k) {
            cudaEvent_t a, b;
            CK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
            cc.in.push_back(a);
            CK(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
            cc.out.push_back(b);
        }
        // the compute stream's earlier work on the staging buffers precedes the uploads
        CK(cudaEventRecord(cc.out[0], c->stream));
        CK(cudaStreamWaitEvent(cc.cs, cc.out[0], 0));
        for (int k = 0; k < nchunk; ++k) {
            const size_t off = (size_t)k * chunk * c->Ng, nb = (size_t)std::min(chunk, nrhs - k * chunk) * c->Ng * 16;
            CK(cudaMemcpyAsync(f.ptr + off, static_cast<const cplx<double>*>(F) + off, nb, cudaMemcpyHostToDevice,
                               cc.cs));
            CK(cudaEventRecord(cc.in[k], cc.cs));
        }
    }
    int rc = HELM_OK;
    helm_stats acc{};
    for (int k = 0; k < nchunk; ++k) {
        const int r0 = k * chunk, nr = std::min(chunk, nrhs - r0);
        const size_t off = (size_t)r0 * c->Ng;
        if (host) CK(cudaStreamWaitEvent(c->stream, cc.in[k], 0));
        if (adjoint) {
            // A^H lam = g  <=>  A conj(lam) = conj(g)  (A^T = A)
            CK(cudaMemcpyAsync(c->bvec + off, f.ptr + off, (size_t)nr * c->Ng * 16, cudaMemcpyDeviceToDevice,
                               c->stream));
            ProfScope ps_(c, HELM_K_KRYLOV, 1);
            launch_conj(c->bvec + off, (int64_t)nr * c->Ng, c->stream);
        } else {
            ProfScope ps_(c, HELM_K_KRYLOV, 1);
            launch_scale_J(c->P, c->gwin, f.ptr + off, c->bvec + off, nr, false, c->stream);
        }
        helm_stats one{};
        const int rci = stationary ? stationary_dev(c, nr, c->bvec + off, u.ptr + off, rtol, maxit, &one)
                                   : gmres_dev(c, nr, c->bvec + off, u.ptr + off, rtol, maxit, &one, restart);
        if (rci != HELM_OK && rci != HELM_ERR_NO_CONVERGENCE) return rci;
        if (rci != HELM_OK) rc = rci;
        acc.iters = std::max(acc.iters, one.iters);
        acc.applications += one.applications;
        acc.resid = std::max(acc.resid, one.resid);
        acc.levels = one.levels;
        acc.solves = one.solves;
        if (adjoint) launch_conj(u.ptr + off, (int64_t)nr * c->Ng, c->stream);
        if (host) {
            CK(cudaEventRecord(cc.out[k], c->stream));
            CK(cudaStreamWaitEvent(cc.cs, cc.out[k], 0));
            CK(cudaMemcpyAsync(static_cast<cplx<double>*>(U) + off, u.ptr + off, (size_t)nr * c->Ng * 16,
                               cudaMemcpyDeviceToHost, cc.cs));
        }
    }
    if (st) *st = acc;
    std::string msg = g_last_error;
    if (host) CK(cudaStreamSynchronize(cc.cs));
    TRY(stage_out(c, U, u, bytes, HELM_MEM_DEVICE));  // waits for the compute stream, checks the device
    if (st) {
        st->t_factor_ms = c->t_factor_ms;
        st->t_solve_ms = now_ms() - t0;
    }
    if (rc != HELM_OK) return fail(rc, msg);
    return HELM_OK;
}

int helm_solve(helm_ctx* c, int nrhs, const void* F, void* U, int mem, double rtol, int maxit,
               helm_stats* st) {
    return solve_common(c, nrhs, F, U, mem, rtol, maxit, st, false);
}

int helm_iterate(helm_ctx* c, int nrhs, const void* F, void* U, int mem, double rtol, int maxit,
                 helm_stats* st) {
    return solve_common(c, nrhs, F, U, mem, rtol, maxit, st, false, true);
}

int helm_adjoint(helm_ctx* c, int nrhs, const void* G, void* L, int mem, double rtol, int maxit,
                 helm_stats* st) {
    return solve_common(c, nrhs, G, L, mem, rtol, maxit, st, true);
}

int helm_gradient(helm_ctx* c, int nsrc, const void* U, const void* L, double* grad, int mem) {
    if (!c || !U || !L || !grad || nsrc < 1) return fail(HELM_ERR_ARG, "bad argument");
    size_t bytes = (size_t)nsrc * c->Ng * 16;
    Staged u, l;
    TRY(stage_in(c, U, bytes, mem, u, 0));
    TRY(stage_in(c, L, bytes, mem, l, 1));
    double* gd = grad;
    bool own = false;
    if (mem == HELM_MEM_HOST) {
        CKM(&gd, c->Ng * 8);
        own = true;
    }
    { ProfScope ps_(c, HELM_K_KRYLOV, 1); launch_gradient(c->P, c->gwin, u.ptr, l.ptr, nsrc, gd, c->stream); }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && own) e = cudaMemcpyAsync(grad, gd, c->Ng * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (own) cudaFree(gd);
    if (e != cudaSuccess) return fail(HELM_ERR_CUDA, cudaGetErrorString(e));
    return HELM_OK;
}

int helm_residual(helm_ctx* c, int nrhs, const void* F, const void* U, void* R, int mem) {
    if (!c || !F || !U || !R || nrhs < 1) return fail(HELM_ERR_ARG, "bad argument");
    size_t bytes = (size_t)nrhs * c->Ng * 16;
    Staged f, u, r;
    TRY(stage_in(c, F, bytes, mem, f, 0));
    TRY(stage_in(c, U, bytes, mem, u, 1));
    TRY(stage_in(c, mem == HELM_MEM_DEVICE ? R : nullptr, bytes, mem, r, 2));
    TRY(ensure_bvec(c, nrhs));
    { ProfScope ps_(c, HELM_K_KRYLOV, 1); launch_scale_J(c->P, c->gwin, f.ptr, c->bvec, nrhs, false, c->stream); }
    { ProfScope ps_(c, HELM_K_KRYLOV, 1); launch_apply_A(c->P, c->stc_d, c->bvec, u.ptr, r.ptr, nrhs, c->stream); }
    CK(cudaGetLastError());
    return stage_out(c, R, r, bytes, mem);
}

int helm_subdomain_solve(helm_ctx* c, int s, int nrhs, const void* R, void* U, int mem) {
    if (!c || !R || !U || nrhs < 1 || s < 0 || s >= c->P.nsub) return fail(HELM_ERR_ARG, "bad argument");
    if (!c->factored) return fail(HELM_ERR_NOT_FACTORED, "call helm_factor first");
    const SubDesc& S = c->subs_h[s];
    const int64_t we = S.win_elems;
    size_t bytes = (size_t)nrhs * we * 16;
    Staged r;
    TRY(stage_in(c, R, bytes, mem, r, 0));
    // a private buffer [rhs][window] in the working precision
    void* wb = nullptr;
    CKM(&wb, (size_t)nrhs * we * elem_size(c));
    std::vector<cplx<double>> host((size_t)nrhs * we);
    CK(cudaMemcpyAsync(host.data(), r.ptr, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->prec == HELM_PREC_F64) {
        CK(cudaMemcpy(wb, host.data(), bytes, cudaMemcpyHostToDevice));
    } else {
        std::vector<cplx<float>> h32(host.size());
        for (size_t i = 0; i < host.size(); ++i) h32[i] = {(float)host[i].re, (float)host[i].im};
        CK(cudaMemcpy(wb, h32.data(), h32.size() * 8, cudaMemcpyHostToDevice));
    }
    Task t{0, s, 0, 0, 0};
    Task* td = nullptr;
    CKM(&td, sizeof(Task));
    CK(cudaMemcpy(td, &t, sizeof(Task), cudaMemcpyHostToDevice));
    launch_one_subdomain_solve(c, td, nrhs, wb, we);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    if (c->prec == HELM_PREC_F64) {
        CK(cudaMemcpy(host.data(), wb, bytes, cudaMemcpyDeviceToHost));
    } else {
        std::vector<cplx<float>> h32(host.size());
        CK(cudaMemcpy(h32.data(), wb, h32.size() * 8, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < host.size(); ++i) host[i] = {h32[i].re, h32[i].im};
    }
    cudaFree(wb);
    cudaFree(td);
    TRY(check_device_error(c));
    if (mem == HELM_MEM_HOST)
        std::memcpy(U, host.data(), bytes);
    else
        CK(cudaMemcpy(U, host.data(), bytes, cudaMemcpyHostToDevice));
    return HELM_OK;
}

int helm_subdomain_solve_noalloc(helm_ctx* c, int s, int nrhs, const void* R, void* U) {
    if (!c || !R || !U || nrhs < 1 || s < 0 || s >= c->P.nsub)
        return fail(HELM_ERR_ARG, "bad argument");
    if (!c->factored) return fail(HELM_ERR_NOT_FACTORED, "call helm_factor first");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != c->device)
        return fail(HELM_ERR_ARG, "helm_subdomain_solve_noalloc: the current device (" + std::to_string(dev) +
                                      ") is not the context's device (" + std::to_string(c->device) + ")");
    const SubDesc& S = c->subs_h[s];
    const size_t need = (size_t)nrhs * S.win_elems * elem_size(c);
    if (need > noalloc_capacity_bytes())
        return fail(HELM_ERR_ARG, "helm_subdomain_solve_noalloc: " + std::to_string(nrhs) +
                                      " right-hand sides on this window need " +
                                      std::to_string(need) + " bytes of scratch; the maximum is " +
                                      std::to_string(noalloc_capacity_bytes()));
    NoAllocArgs a;
    a.f64 = c->prec == HELM_PREC_F64;
    a.sub = s;
    a.nrhs = nrhs;
    a.win_elems = S.win_elems;
    a.R = static_cast<const cplx<double>*>(R);
    a.U = static_cast<cplx<double>*>(U);
    a.stream = c->stream;
    a.solve = noalloc_solve_cb;
    a.ctx = c;
    CK(noalloc_subdomain_solve(a));
    CK(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int helm_window_info(helm_ctx* c, int s, int64_t lo[3], int64_t hi[3]) {
    if (!c || s < 0 || s >= c->P.nsub || !lo || !hi) return fail(HELM_ERR_ARG, "bad argument");
    for (int a = 0; a < 3; ++a) {
        lo[a] = c->subs_h[s].lo[a];
        hi[a] = c->subs_h[s].hi[a];
    }
    return HELM_OK;
}

int helm_problem_info(helm_ctx* c, int64_t* nsub, int64_t N[3]) {
    if (!c) return fail(HELM_ERR_ARG, "null context");
    if (nsub) *nsub = c->P.nsub;
    if (N)
        for (int a = 0; a < 3; ++a) N[a] = c->P.N[a];
    return HELM_OK;
}

int64_t helm_device_bytes(helm_ctx* c) { return c ? (int64_t)c->dev_bytes : 0; }

int helm_release(helm_ctx* c) {
    if (!c) return fail(HELM_ERR_ARG, "null context");
    CK(cudaStreamSynchronize(c->stream));  // nothing queued may still use what is freed
    auto drop = [&](auto*& p, size_t bytes) {
        if (p) {
            cudaFree(p);
            c->dev_bytes -= bytes;
        }
        p = nullptr;
    };
    drop(c->fac, c->fac_bytes);
    drop(c->ufac, c->ufac_bytes);
    drop(c->ufac_off, c->subs_h.size() * sizeof(int64_t));
    drop(c->ascale_d, c->inva_count * sizeof(int));
    const size_t wb = (size_t)c->cap_rhs * c->buf_per_rhs * elem_size(c);
    drop(c->buf, wb);
    drop(c->bsrc, wb);
    drop(c->bvec, (size_t)c->cap_vec_rhs * c->Ng * 16);
    for (auto*& p : c->gm) drop(p, (size_t)c->gm_rhs * c->Ng * 16);
    for (int i = 0; i < 3; ++i) drop(c->stage_d[i], c->stage_cap[i]);
    c->gm.clear();
    c->ufac_bytes = 0;
    c->cap_rhs = c->cap_vec_rhs = c->gm_rhs = 0;
    for (auto& s : c->stage_cap) s = 0;
    c->umma_twist = false;
    c->umma_mt = 0;
    c->panel_pick.clear();
    c->factored = false;
    CK(cudaGetLastError());
    return HELM_OK;
}

int helm_profile_reset(helm_ctx* c) {
    if (!c) return fail(HELM_ERR_ARG, "null context");
    CK(cudaStreamSynchronize(c->stream));
    resolve_profile(c);
    c->prof = helm_profile{};
    return HELM_OK;
}

int helm_profile_get(helm_ctx* c, helm_profile* out) {
    if (!c || !out) return fail(HELM_ERR_ARG, "bad argument");
    CK(cudaStreamSynchronize(c->stream));
    resolve_profile(c);
    *out = c->prof;
    return HELM_OK;
}

void helm_destroy(helm_ctx* c) {
    if (!c) return;
    void* ptrs[] = {c->ufac, c->ufac_off, c->subs_d, c->g_alpha, c->m64, c->m32, c->an64, c->af64, c->an32, c->af32,
                    c->Pv64, c->inva64, c->Pv32, c->inva32, c->tab64, c->tab32, c->box_of,
                    c->fac, c->err_d, c->tasks_d, c->inc_d, c->gnode_d, c->gblk_d, c->node_buf_d, c->buf,
                    c->bvec,
                    c->small_d, c->partial_d, c->vptr_d, c->zptr_d, c->ascale_d, c->bsrc,
                    c->stc_d, c->stage_d[0], c->stage_d[1], c->stage_d[2]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto* p : c->gm) cudaFree(p);
    if (c->stream) cudaStreamSynchronize(c->stream);
    resolve_profile(c);
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->cstream) cudaStreamDestroy(c->cstream);
    delete c;
}

const char* helm_strerror(int code) {
    switch (code) {
        case HELM_OK: return "ok";
        case HELM_ERR_ARG: return "invalid argument";
        case HELM_ERR_OOM: return "out of device memory";
        case HELM_ERR_NOT_FACTORED: return "not factored";
        case HELM_ERR_NO_CONVERGENCE: return "GMRES did not converge";
        case HELM_ERR_TIMEOUT: return "device wait timed out";
        case HELM_ERR_CUDA: return "CUDA error";
        case HELM_ERR_NUMERIC: return "numerical breakdown in a factor";
        default: return "unknown error";
    }
}

const char* helm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
