// Internal types shared by the libhelm translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/helm.h"

namespace helm {

// ----------------------------------------------------------------------------- complex
template <typename T>
struct cplx {
    T re, im;
};
template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };

template <typename T>
__host__ __device__ __forceinline__ cplx<T> mk(T r, T i) { return cplx<T>{r, i}; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> cneg(cplx<T> a) { return {-a.re, -a.im}; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return {a.re, -a.im}; }
template <typename T>
__host__ __device__ __forceinline__ T cabs2(cplx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> cinv(cplx<T> a) {
    T s = T(1) / (a.re * a.re + a.im * a.im);
    return {a.re * s, -a.im * s};
}
// acc += a * b
template <typename T>
__host__ __device__ __forceinline__ void cfma(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
template <typename T, typename U>
__host__ __device__ __forceinline__ cplx<T> ccast(cplx<U> a) { return {T(a.re), T(a.im)}; }

// ----------------------------------------------------------------------------- window
// A box-shaped window of the full grid with its own PML coefficients: the
// global problem (lo = 0, n = N) or one subdomain problem P_{Omega_ij}.
// alpha_node[a][i] = alpha_a at node lo[a]+i, alpha_face[a][i] = alpha_a at the
// face between nodes lo[a]+i-1 and lo[a]+i (i = 0..n[a]).
template <typename T>
struct Win {
    int lo[3];
    int n[3];
    const cplx<T>* alpha_node[3];
    const cplx<T>* alpha_face[3];
};

// The 2*ndim+1 coefficients of row k of the J-multiplied PML operator:
// (A u)_k = diag u_k + sum_a cp[a] u_{k+e_a} + cm[a] u_{k-e_a}
//   cp[a] = prod_{b!=a} alpha_b(node) / (h^2 alpha_a(face k_a+1/2)),
//   cm[a] likewise with the face k_a-1/2,
//   diag  = omega^2 m J - sum_a (cp[a] + cm[a]),  J = prod_b alpha_b(node).
template <typename T>
struct Stencil {
    cplx<T> diag;
    cplx<T> cp[3], cm[3];
};

template <typename T>
__device__ __forceinline__ Stencil<T> stencil_at(const Win<T>& w, int ndim, const int x[3],
                                                 T inv_h2, T omega2, T m) {
    cplx<T> an[3];
    for (int a = 0; a < 3; ++a) an[a] = (a < ndim) ? w.alpha_node[a][x[a]] : mk<T>(1, 0);
    Stencil<T> s;
    cplx<T> J = an[0] * an[1] * an[2];
    cplx<T> sum = mk<T>(0, 0);
    for (int a = 0; a < 3; ++a) {
        if (a >= ndim) {
            s.cp[a] = s.cm[a] = mk<T>(0, 0);
            continue;
        }
        cplx<T> P = mk<T>(inv_h2, 0);
        for (int b = 0; b < ndim; ++b)
            if (b != a) P = P * an[b];
        s.cp[a] = P * cinv(w.alpha_face[a][x[a] + 1]);
        s.cm[a] = P * cinv(w.alpha_face[a][x[a]]);
        sum = sum + s.cp[a] + s.cm[a];
    }
    s.diag = (omega2 * m) * J - sum;
    return s;
}

// ----------------------------------------------------------------------------- subdomains
struct SubDesc {
    int lo[3], hi[3];          // window node range (global, hi exclusive)
    int box_lo[3], box_hi[3];  // box node range (global)
    int nw[3];                 // window sizes (nw[2] = 1 in 2D)
    int ib[3];                 // box index per axis
    int nblk;                  // nodes per block (line in 2D, plane in 3D)
    int nbp;                   // nblk padded to a multiple of 32
    int nlines;                // blocks (window extent along the slowest axis)
    int64_t alpha_off[3];      // offset of this window's node alphas per axis
    int64_t face_off[3];       // offset of this window's face alphas per axis
    int64_t fac_off;           // offset (elements of T) of this subdomain's factors
    int64_t coup_off;          // offset of Pv (nblk) in the coupling arrays
    int64_t inva_off;          // offset of 1/alpha_slow(face) (nlines+1)
    int64_t win_elems;         // nodes in the window
};

// One (sweep, subdomain) solve of a dependency level, with its incoming
// transferred sources [in_off, in_off + in_cnt).
struct Task {
    int sweep;
    int sub;
    int in_off, in_cnt;
    int64_t buf_off;  // element offset (complex) of this node's window buffer per RHS block
};

// Incoming transferred source: Psi_{dir; sender}(u^{l_src}_{sender}).
struct Incoming {
    int dir[3];
    int sender;
    int64_t sender_buf_off;
};

// ----------------------------------------------------------------------------- kernels
struct DevProblem {
    int ndim;
    int N[3];
    int d;                  // overlap cells
    int nsub;
    int nb[3];
    double h, omega;
};

void launch_factor_f32(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                       const float* m32, const cplx<float>* an, const cplx<float>* af,
                       float* fac, int* err, cudaStream_t st);
// Twisted factors of lines nlines/2 .. nlines-1 (k_factor.cu) into fac2; reads
// the standard factors of line nlines/2 - 1 from fac.
void launch_factor_twist_f32(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                             const float* m32, const cplx<float>* an, const cplx<float>* af,
                             const float* fac, float* fac2, int* err, cudaStream_t st);
void launch_factor_f64(const SubDesc* subs, int nsub, int nbp_max, const DevProblem& P,
                       const double* m64, const cplx<double>* an, const cplx<double>* af,
                       double* fac, int* err, cudaStream_t st);

// Error reporting and wait bounds of the solve kernels.  Every spin-wait in
// them is bounded.  An ordinary wait (a copy, an MMA commit, a cluster
// handshake the kernel needs to make progress) gives up after `polls` polls
// (0: at once); the kernel then writes 2 to *err, stops issuing work and
// drains what it already started.  The drain waits always use kDrainPolls,
// so no CTA releases shared memory or TMEM while a copy or MMA still targets it.
constexpr uint32_t kDrainPolls = 1u << 22;
constexpr uint32_t kDefaultWaitPolls = 1u << 22;
struct DevStatus {
    int* err;        // device error word: 1 = numerical breakdown, 2 = a wait expired
    uint32_t polls;  // polls of each ordinary wait
};

// buf: y, then u of every solve (read by the transfers and the assembly);
// bsrc: the local sources b the gather wrote (same layout), read by the solve.
template <typename T>
void launch_solve(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                  int panel, const T* fac, const cplx<T>* Pv, const cplx<T>* inva, cplx<T>* buf,
                  const cplx<T>* bsrc, int64_t buf_rhs_stride, DevStatus ds, cudaStream_t st);

// Tensor-core (TF32 mma, FP32 accumulate) variant for complex64 factors.
void launch_solve_tc(const Task* tasks, int ntask, const SubDesc* subs, int nbp_max, int nrhs,
                     int panel, const float* fac, const cplx<float>* Pv, const cplx<float>* inva,
                     cplx<float>* buf, const cplx<float>* bsrc, int64_t buf_rhs_stride, DevStatus ds,
                     cudaStream_t st);
void launch_round_tf32(float* x, int64_t count, cudaStream_t st);

// tcgen05 (5th-generation tensor core) subdomain solve, k_solve_umma.cu.  The
// factors are repacked into 128-byte-swizzled K-major images, the block rows
// split evenly over the umma_tiles(n) CTAs of a cluster.
int umma_tiles(int nblk_max);
bool umma_supported(int nblk_max);
int64_t umma_factor_bytes(const SubDesc& S, int mt);
void launch_repack_umma(const SubDesc* subs_d, const std::vector<SubDesc>& subs_h, int mt,
                        const float* fac, const float* fac2, const int64_t* dst_off_d, float* dst,
                        cudaStream_t st);  // fac2: twisted factors of lines >= nlines/2, or null
// Twisted (two-ended) tcgen05 solve: one 2-CTA cluster per (task, panel of 8
// RHS), top and bottom halves of the lines, all rows per CTA (n <= 256 in two
// M = 128 tiles, or n <= 384 in three with f16; nlines >= 4); factors repacked with one slice (CR = 1) from the twisted factors.
// With f16 the image is FP16 (K chunks of 64) with per-line power-of-two
// scales ascale[inva_off + line] (launch_line_scales, launch_repack_f16).
bool twist_supported(int nblk_max, int nlines_min, int nlines_max, bool f16);
int64_t twist_f16_factor_bytes(const SubDesc& S);
void launch_line_scales(const SubDesc* subs_d, int nsub, int max_lines, const float* fac, const float* fac2,
                        int* ascale, cudaStream_t st);
void launch_repack_f16(const SubDesc* subs_d, const std::vector<SubDesc>& subs_h, const float* fac,
                       const float* fac2, const int* ascale, const int64_t* dst_off_d, void* dst,
                       cudaStream_t st);
void launch_solve_twist(const Task* tasks, int ntask, const SubDesc* subs, int nblk_max, int nlines_max, int nrhs,
                        const void* afac, const int64_t* afac_off, const int* ascale, bool f16,
                        const cplx<float>* Pv, const cplx<float>* inva, cplx<float>* buf,
                        const cplx<float>* bsrc, int64_t rstride, DevStatus ds, cudaStream_t st);
void launch_solve_umma(const Task* tasks, int ntask, const SubDesc* subs, int nblk_max, int nrhs,
                       int panel, const float* afac, const int64_t* afac_off,
                       const cplx<float>* Pv, const cplx<float>* inva, cplx<float>* buf,
                       const cplx<float>* bsrc, int64_t rstride, DevStatus ds, cudaStream_t st);

// Work list of the gather: per task (in level order) the window nodes that
// are ever written -- the first sweep's box, and every node some incoming
// transfer's strip reaches -- in window order, each with the transfers that
// reach it (bit i: the task's i-th incoming transfer; bit 31: in the first
// sweep's box).  Blocks take up to kGB consecutive nodes of one task.
// launch_gather reads the senders' solutions in buf and writes the local
// sources into bsrc.
constexpr int kGB = 128;
struct GNode {
    uint32_t k;     // window-linear node index
    uint32_t mask;
};
struct GBlock {
    int task;       // index into the level-ordered task array
    int cnt;        // nodes (<= kGB)
    int64_t node0;  // first node in the GNode array
};
template <typename T, typename VB>
void launch_gather(const GBlock* blocks, int nblocks, const GNode* nodes, const Task* tasks,
                   const SubDesc* subs, const Incoming* inc, const DevProblem& P, const T* m,
                   const cplx<T>* an, const cplx<T>* af, const T* beta_tab, const VB* b, int nrhs,
                   const cplx<T>* buf, cplx<T>* bsrc, int64_t rstride, cudaStream_t st);

// u_DDM into U: complex128, or float-float (float4 per entry) for the Krylov work vectors
template <typename T, typename VU>
void launch_assemble(const DevProblem& P, const SubDesc* subs, const int* box_of, const int64_t* node_buf,
                     int nsweeps, const T* beta_tab, const cplx<T>* buf, int64_t rstride, int nrhs, VU* U,
                     cudaStream_t st);

// global FP64 kernels
void launch_scale_J(const DevProblem& P, const Win<double>& g, const cplx<double>* f,
                    cplx<double>* b, int nrhs, bool conj_in, cudaStream_t st);
void launch_stencil_ff(const DevProblem& P, const Win<double>& g, const double* m, float4* stc,
                       cudaStream_t st);
// The GMRES work vectors (w, V_i, Z_i) are float-float, one float4 (re.hi,
// re.lo, im.hi, im.lo) per complex entry, so the Krylov kernels neither split
// nor join doubles; the caller's complex128 arrays (b, x) are split on load
// and joined on store.
// r = b - A u (b may be null: r = -A u); u, r complex128 or float-float
template <typename VU, typename VR>
void launch_apply_A(const DevProblem& P, const float4* stc, const cplx<double>* b, const VU* u, VR* r, int nrhs,
                    cudaStream_t st);
template <typename VV>
void launch_norms2(const VV* v, int64_t n, int nrhs, cplx<double>* out, cplx<double>* partial, int nblk,
                   cudaStream_t st);  // out[c] = |v[c]|^2
// fused over nv float-float vectors given as a device array of pointers (nv <= 64)
void launch_mdots(const float4* const* V, int nv, const float4* w, int64_t n, int nrhs, cplx<double>* out,
                  cplx<double>* partial, int nblk, cudaStream_t st);  // out[i*nrhs+c] = <V_i[c], w[c]>
int mdots_launches(int nv);  // kernel launches launch_mdots makes for nv vectors
template <typename VW>
void launch_mcombo(VW* w, const float4* const* V, int nv, const cplx<double>* coef, int64_t n, int nrhs,
                   double sign, cudaStream_t st);  // w[c] += sign * sum_i coef[i*nrhs+c] V_i[c]
// w[c] += sum_i coef[i*nrhs+c] U_i[c] fused with, of the updated w, the dots
// out[i*nrhs+c] = <U_i[c], w[c]> (want_dots) or the squared norms out[c];
// 1 <= nv <= kComboDotsMax, else cudaErrorInvalidValue and nothing launched
constexpr int kComboDotsMax = 8;
cudaError_t launch_combo_dots(float4* w, const float4* const* U, int nv, const cplx<double>* coef, int64_t n,
                              int nrhs, bool want_dots, cplx<double>* out, cplx<double>* partial, int nblk,
                              cudaStream_t st);
  // v[c] = src[c] * s[c]
void launch_conj(cplx<double>* v, int64_t count, cudaStream_t st);
// w = b converted to float-float (float4 per entry), count entries.
void launch_to_ff(const cplx<double>* b, float4* w, int64_t count, cudaStream_t st);
void launch_gradient(const DevProblem& P, const Win<double>& g, const cplx<double>* U,
                     const cplx<double>* L, int nsrc, double* grad, cudaStream_t st);

// Subdomain solve inside a static device scratch array (k_noalloc.cu).  The
// solve itself is queued by `solve` (the context's kernel choice, in place on
// the window buffer it is given, allocating nothing).
struct NoAllocArgs {
    bool f64;
    int sub, nrhs;
    int64_t win_elems;
    const cplx<double>* R;
    cplx<double>* U;
    cudaStream_t stream;
    void (*solve)(void* ctx, const Task* task, int nrhs, void* wb, int64_t win_elems);
    void* ctx;
};
size_t noalloc_capacity_bytes();
cudaError_t noalloc_subdomain_solve(const NoAllocArgs& a);

}  // namespace helm
