// Subdomain solves on the 5th-generation tensor cores: tcgen05.mma (kind::tf32)
// with TMEM accumulators, operands in shared memory fed by the bulk-copy engine.
//
// Recurrence (block-Thomas, k_factor.cu): forward y_j = D_j (b_j - a_j y_{j-1}),
// backward u_j = y_j - D_j (c_j u_{j+1}).  Each block product D_j R is one real
// GEMM  Y[M=n rows][N=2*PG] = A[M][K] B[K][N]  with
//   K index k = 2q + part:   A[p][2q+part] = part ? Im D(p,q) : Re D(p,q)
//   N index n = 2c + w:      B[2q][2c] = Re r, B[2q+1][2c] = -Im r,
//                            B[2q][2c+1] = Im r, B[2q+1][2c+1] = Re r
// so Y[p][2c] = Re y_pc and Y[p][2c+1] = Im y_pc.
//
// Layouts (all K-major with the 128-byte swizzle: rows of 32 TF32 values, the
// 16-byte chunk c of row r stored at chunk c ^ (r % 8), 8-row groups 1024 B apart):
//   * A: the factors are repacked once (repack_umma_kernel) into the exact
//     shared-memory image, [line][K chunk of 32][M tile of 128 rows][16 KB], so a
//     whole K chunk of every M tile is one contiguous span for cp.async.bulk.
//   * B: built in shared memory by the epilogue threads, [K chunk][N rows][128 B].
//
// Roles (one CTA per (task, panel of PG right-hand sides, 128-row M tile);
// the CTAs of the M tiles of a block form a thread-block cluster, N = 2 PG):
//   warps 0-3   epilogue: thread = one block row p; reads its row of the
//               accumulator from TMEM (tcgen05.ld), stores y or u, and writes
//               row p of the next B into every CTA of the cluster (DSMEM)
//   warp 4      producer: bulk copies of this CTA's A tile, chunk by chunk,
//               into a ring deep enough to hold most of a line
//   warp 5      TMEM allocation; lane 0 issues the MMAs and commits
// Handshakes are mbarriers: full/empty per stage (TMA bytes / tcgen05.commit),
// acc_full per step (tcgen05.commit), b_ready per step (the epilogue threads
// of every CTA of the cluster, remote arrivals with release semantics).
// Every wait is bounded; on expiry the CTA raises the device error word, each
// role leaves its loop, outstanding copies and MMAs are drained (bounded),
// and TMEM is freed before the CTA exits.
#include <algorithm>

#include "helm_internal.h"

namespace helm {

namespace {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mb_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mb_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// Bounded wait with cluster-scope acquire: pairs with remote release arrivals.
__device__ __forceinline__ bool mb_wait_cluster(uint32_t bar, uint32_t parity, uint32_t limit) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: start address,
// leading byte offset (unused for this layout, 1), stride byte offset 1024
// (8 rows x 128 B), descriptor version 1, layout type 2 (128B swizzle).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// Instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr uint32_t kWait = kDrainPolls;
constexpr int kChunkK = 32;        // K values per 128-byte row
constexpr int kTileBytes = 128 * 128;  // 128 rows x 128 B

}  // namespace

// Bytes of one line's repacked A for a block of n rows stored with MT M tiles
// of 128 rows (every subdomain of a context uses the same MT):
// ceil(2*roundup4(n)/32) K chunks x MT tiles x 16 KB.
__host__ __device__ inline int64_t umma_line_bytes(int n, int MT, int* nkc) {
    const int n4 = (n + 3) & ~3;
    const int kc = (2 * n4 + kChunkK - 1) / kChunkK;
    if (nkc) *nkc = kc;
    return (int64_t)kc * MT * kTileBytes;
}

// Repack the column-major factors of every subdomain (k_factor.cu layout) into
// the swizzled tile image, rounding to TF32.  One thread per output float.
__global__ void repack_umma_kernel(const SubDesc* __restrict__ subs, const float* __restrict__ fac,
                                   const int64_t* __restrict__ dst_off, float* dst, int sub, int mt) {
    const SubDesc& S = subs[sub];
    int nkc;
    const int64_t lb = umma_line_bytes(S.nblk, mt, &nkc) / 4;  // floats per line
    const int64_t total = lb * S.nlines;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int j = (int)(i / lb);
    int64_t rem = i % lb;
    const int kc = (int)(rem / (mt * 4096));
    rem %= (mt * 4096);
    const int tile = (int)(rem / 4096);
    const int off = (int)(rem % 4096);  // float offset in the 16 KB tile image
    const int r = off / 32;             // row in tile
    const int pos = off % 32;           // float position within the 128-byte row
    const int chunk = (pos / 4) ^ (r % 8);
    const int kk = chunk * 4 + (pos % 4);  // logical K within the chunk
    const int p = tile * 128 + r;
    const int k = kc * kChunkK + kk;
    const int q = k >> 1, part = k & 1;
    float v = 0.f;
    if (p < S.nblk && q < S.nblk) {
        const float* D = fac + S.fac_off + (int64_t)j * 2 * S.nbp * S.nbp;
        v = D[(int64_t)q * 2 * S.nbp + part * S.nbp + p];
    }
    dst[dst_off[sub] / 4 + i] = __uint_as_float(to_tf32(v));  // dst_off in bytes
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t map_peer(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_v2(uint32_t addr, float a, float b) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void mb_arrive_cluster(uint32_t addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One CTA per (task, panel of PG right-hand sides, 128-row M tile); the CTAs
// of the M tiles of one block form a cluster of CR (1 or 2).  Each CTA streams
// and multiplies only its own tile of D_j, holds the whole K extent of B, and
// its epilogue writes the B rows of its block rows into every CTA of the
// cluster (distributed shared memory) and arrives on every CTA's b_ready.
// B is double-buffered: a peer may be one step ahead.
constexpr int kIssuers = 4;  // MMA-issuing warps; K chunks are dealt round-robin to them

template <int PG>
__global__ void __launch_bounds__(32 * (5 + kIssuers)) solve_umma_kernel(
    const Task* __restrict__ tasks, const SubDesc* __restrict__ subs, int nrhs, int CR,
    const float* __restrict__ afac, const int64_t* __restrict__ afac_off,
    const cplx<float>* __restrict__ Pv, const cplx<float>* __restrict__ inva, cplx<float>* buf,
    int64_t rstride, int nstage, DevStatus ds) {
    constexpr int kN = 2 * PG;              // real columns
    constexpr int kBChunkBytes = kN * 128;  // B rows of one K chunk
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t rank = CR > 1 ? cluster_rank() : 0;
    const Task tk = tasks[blockIdx.x / CR];
    const SubDesc& S = subs[tk.sub];
    const int n = S.nblk, nl = S.nlines;
    int nkc;
    const int64_t line_bytes = umma_line_bytes(n, CR, &nkc);
    const int NS = nstage;
    const uint32_t bbuf_bytes = (uint32_t)(nkc * kBChunkBytes);

    // shared layout (1024-aligned): stages | B[2] | barriers | tmem slot | flag
    const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - su32(smem_raw));
    const uint32_t stage0 = base;
    const uint32_t b0 = stage0 + NS * kTileBytes;
    float* bgen = reinterpret_cast<float*>(gbase + NS * kTileBytes);
    const uint32_t bars = b0 + 2 * bbuf_bytes;
    uint64_t* bars_g = reinterpret_cast<uint64_t*>(gbase + NS * kTileBytes + 2 * bbuf_bytes);
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (NS + s); };
    const uint32_t acc_full = bars + 8u * (2 * NS);
    // b_ready of step s is barrier s & 1: arrivals of consecutive steps never
    // share a phase (a count-based phase cannot tell the steps apart, and a
    // peer CTA may arrive for step s+1 before this CTA's last step-s arrival)
    auto b_ready = [&](int step) { return bars + 8u * (2 * NS + 1 + (step & 1)); };
    const uint32_t drain = bars + 8u * (2 * NS + 3);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars_g + 2 * NS + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nsteps = 2 * nl - 1;
    const int total_chunks = nsteps * nkc;
    // one accumulator of kN columns per issuer
    constexpr uint32_t kCols = kIssuers * kN <= 32 ? 32 : kIssuers * kN <= 64 ? 64 :
                               kIssuers * kN <= 128 ? 128 : 256;

    if (tid == 0) {
        *abort_flag = 0;
        for (int s = 0; s < NS; ++s) {
            mb_init(full(s), 1);
            mb_init(empty(s), 1);
        }
        mb_init(acc_full, kIssuers);
        mb_init(b_ready(0), 128 * CR);  // every epilogue thread of every CTA of the cluster
        mb_init(b_ready(1), 128 * CR);
        mb_init(drain, kIssuers);  // completes once every issuer's MMAs have
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (uint32_t i = tid; i < 2 * bbuf_bytes / 4; i += blockDim.x) bgen[i] = 0.f;
    {
        float* sg = reinterpret_cast<float*>(gbase);
        for (uint32_t i = tid; i < (uint32_t)NS * kTileBytes / 4; i += blockDim.x) sg[i] = 0.f;
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    if (CR > 1) cluster_sync();  // peers' barriers are initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 4) {
        // ====================================================== producer
        if (lane == 0) {
            const char* abase = reinterpret_cast<const char*>(afac) + afac_off[tk.sub];
            int rows = n - (int)rank * 128;
            rows = rows < 8 ? 8 : ((rows + 7) & ~7);
            if (rows > 128) rows = 128;
            const uint32_t copy_bytes = (uint32_t)(rows * 128);
            int issued = 0;
            for (int i = 0; i < total_chunks; ++i) {
                const int s = i % NS;
                if (i >= NS && !mb_wait(empty(s), (uint32_t)(((i / NS) - 1) & 1), ds.polls)) {
                    atomicExch(ds.err, 2);
                    *abort_flag = 1;
                }
                if (*abort_flag) break;
                const int step = i / nkc, kc = i % nkc;
                const int j = step < nl ? step : 2 * nl - 2 - step;
                mb_expect_tx(full(s), copy_bytes);
                bulk_g2s(stage0 + s * kTileBytes,
                         abase + (int64_t)j * line_bytes + ((int64_t)kc * CR + rank) * kTileBytes,
                         copy_bytes, full(s));
                issued = i + 1;
            }
            for (int i = (issued > NS ? issued - NS : 0); i < issued; ++i)
                mb_wait(full(i % NS), (uint32_t)((i / NS) & 1), kWait);
        }
    } else if (warp >= 5 && warp < 5 + kIssuers) {
        // ====================================================== MMA issuers
        // issuer q takes the K chunks kc = q, q + kIssuers, ... of every line
        // into its own accumulator (columns q*kN ...), so the per-instruction
        // issue latency of the chunks overlaps across warps
        const int q = warp - 5;
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(128, kN);
            const uint32_t dacc = tmem + (uint32_t)(q * kN);
            for (int step = 0; step < nsteps && !*abort_flag; ++step) {
                if (!mb_wait_cluster(b_ready(step), (uint32_t)((step >> 1) & 1), ds.polls)) {
                    atomicExch(ds.err, 2);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint64_t bdesc0 = desc_sw128(b0 + (step & 1) * bbuf_bytes);
                bool first = true;
                for (int kc = q; kc < nkc; kc += kIssuers) {
                    const int ci = step * nkc + kc;
                    const int s = ci % NS;
                    if (!mb_wait(full(s), (uint32_t)((ci / NS) & 1), ds.polls)) {
                        atomicExch(ds.err, 2);
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t adesc = desc_sw128(stage0 + s * kTileBytes);
                    const uint64_t bdesc = bdesc0 + (uint64_t)(kc * (kBChunkBytes >> 4));
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_tf32(dacc, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk), idesc,
                                  (first && kk == 0) ? 0u : 1u);
                    first = false;
                    umma_commit(empty(s));
                }
                if (*abort_flag) break;
                // (an issuer without a chunk -- K shorter than kIssuers chunks -- commits
                // nothing pending; the epilogue never reads its accumulator)
                umma_commit(acc_full);
            }
            umma_commit(drain);
            mb_wait(drain, 0u, kWait);
        }
    } else {
        // ====================================================== epilogue (warps 0-3)
        const int p = (int)rank * 128 + warp * 32 + lane;  // owned block row
        const bool rv = p < n;
        const int n4 = (n + 3) & ~3;
        const cplx<float> pvp = rv ? Pv[S.coup_off + p] : mk<float>(0, 0);
        const cplx<float>* ia = inva + S.inva_off;
        cplx<float>* V = buf + tk.buf_off;
        const int c0 = blockIdx.y * PG;
        int ncol = nrhs - c0;
        if (ncol > PG) ncol = PG;
        const int k0 = 2 * p;  // B rows k0 (Re column) and k0+1 (Im column)
        const int kcb = k0 / kChunkK, kkb = k0 % kChunkK;
        // byte offset of B[row][k0] within a buffer (k0, k0+1 adjacent)
        auto boff = [&](int row) -> uint32_t {
            const int chunk = (kkb / 4) ^ (row % 8);
            return (uint32_t)(kcb * kBChunkBytes + row * 128 + chunk * 16 + (kkb % 4) * 4);
        };
        uint32_t peer_b[2] = {b0, b0}, peer_ready[2] = {b_ready(0), b_ready(0)};
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (r < CR) {
                peer_b[r] = map_peer(b0, (uint32_t)r);
                peer_ready[r] = map_peer(b_ready(0), (uint32_t)r);  // b_ready(1) is 8 bytes on
            }
        // write B rows k0, k0+1 for right-hand side c into buffer bb of every CTA
        auto put_b = [&](int bb, int c, cplx<float> v) {
            const float re = __uint_as_float(to_tf32(v.re)), im = __uint_as_float(to_tf32(v.im));
            const float nim = __uint_as_float(to_tf32(-v.im));
            const uint32_t o0 = (uint32_t)bb * bbuf_bytes + boff(2 * c);
            const uint32_t o1 = (uint32_t)bb * bbuf_bytes + boff(2 * c + 1);
#pragma unroll
            for (int r = 0; r < 2; ++r)
                if (r < CR) {
                    st_cluster_v2(peer_b[r] + o0, re, nim);  // row 2c:   Re r, -Im r
                    st_cluster_v2(peer_b[r] + o1, im, re);   // row 2c+1: Im r,  Re r
                }
        };
        auto signal = [&](int step) {  // B of `step` is written everywhere
            asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
            tc_fence_before();
#pragma unroll
            for (int r = 0; r < 2; ++r)
                if (r < CR) mb_arrive_cluster(peer_ready[r] + 8u * (step & 1));
        };
        // operand needed after the product of step s: b_{j+1} (forward line j)
        // or y_j (backward line j); loaded one whole step ahead
        auto operand_line = [&](int step) -> int {
            if (step >= nsteps) return -1;
            if (step < nl) return step + 1 < nl ? step + 1 : -1;
            return 2 * nl - 2 - step;
        };
        auto load_operand = [&](int step, cplx<float> (&dst)[PG]) {
            const int jj = operand_line(step);
#pragma unroll
            for (int c = 0; c < PG; ++c)
                dst[c] = (rv && c < ncol && jj >= 0) ? V[(int64_t)(c0 + c) * rstride + (int64_t)jj * n + p]
                                                     : mk<float>(0, 0);
        };
        cplx<float> pre[PG], pre_next[PG], outv[PG];
#pragma unroll
        for (int c = 0; c < PG; ++c) {
            cplx<float> b = (rv && c < ncol) ? V[(int64_t)(c0 + c) * rstride + p] : mk<float>(0, 0);
            if (p < n4) put_b(0, c, b);
        }
        load_operand(0, pre);
        signal(0);
        for (int step = 0; step < nsteps; ++step) {
            const bool fwd = step < nl;
            const int j = fwd ? step : 2 * nl - 2 - step;
            load_operand(step + 1, pre_next);
            bool bad = *abort_flag || !mb_wait(acc_full, (uint32_t)(step & 1), ds.polls);
            if (__any_sync(0xffffffffu, bad)) {  // warp-uniform before the collective load
                atomicExch(ds.err, 2);
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            float acc[kN];
#pragma unroll
            for (int e = 0; e < kN; ++e) acc[e] = 0.f;
#pragma unroll
            for (int iq = 0; iq < kIssuers; ++iq) {
                if (iq >= nkc) break;  // issuers without a chunk hold no partial sum
#pragma unroll
                for (int q = 0; q < kN / 16; ++q) {
                    float part[16];
                    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + iq * kN + 16 * q, part);
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[16 * q + e] += part[e];
                }
            }
            cplx<float> coup = mk<float>(0, 0);
            if (rv) {
                if (fwd && j + 1 < nl) coup = pvp * ia[j + 1];   // a_{j+1}
                else if (fwd) coup = pvp * ia[nl - 1];            // c_{nl-2}
                else if (j > 0) coup = pvp * ia[j];               // c_{j-1}
            }
            const int nb = (step + 1) & 1;
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                const cplx<float> y = mk<float>(acc[2 * c], acc[2 * c + 1]);
                outv[c] = fwd ? y : pre[c] - y;
                cplx<float> nbv = mk<float>(0, 0);
                if (rv) nbv = (fwd && j + 1 < nl) ? pre[c] - coup * outv[c] : coup * outv[c];
                if (step + 1 < nsteps && p < n4) put_b(nb, c, nbv);
            }
            if (step + 1 < nsteps) signal(step + 1);
            // global stores after the release-arrive, so it does not wait for them
#pragma unroll
            for (int c = 0; c < PG; ++c) {
                if (rv && c < ncol) V[(int64_t)(c0 + c) * rstride + (int64_t)j * n + p] = outv[c];
                pre[c] = pre_next[c];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (CR > 1) cluster_sync();  // no CTA leaves while a peer may still write into it
    tc_fence_after();
    if (warp == 5)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
}

void launch_repack_umma(const SubDesc* subs_d, const std::vector<SubDesc>& subs_h, int mt,
                        const float* fac, const int64_t* dst_off_d, float* dst, cudaStream_t st) {
    for (size_t s = 0; s < subs_h.size(); ++s) {
        const int64_t floats = umma_line_bytes(subs_h[s].nblk, mt, nullptr) / 4 * subs_h[s].nlines;
        repack_umma_kernel<<<(unsigned)((floats + 255) / 256), 256, 0, st>>>(subs_d, fac, dst_off_d,
                                                                             dst, (int)s, mt);
    }
}

int umma_tiles(int nblk_max) { return (nblk_max + 127) / 128; }

int64_t umma_factor_bytes(const SubDesc& S, int mt) { return umma_line_bytes(S.nblk, mt, nullptr) * S.nlines; }

template <int PG>
static void launch_pg(const Task* tasks, int ntask, const SubDesc* subs, int CR, int nkc_max,
                      int nrhs, const float* afac, const int64_t* afac_off, const cplx<float>* Pv,
                      const cplx<float>* inva, cplx<float>* buf, int64_t rstride, DevStatus ds,
                      cudaStream_t st) {
    const size_t bbuf = (size_t)nkc_max * 2 * PG * 128;
    const size_t fixed = 2 * bbuf + 8 * 64 + 64 + 1024;  // B[2], barriers, slots, alignment
    int ns = (int)std::min<size_t>(16, (224 * 1024 - fixed) / kTileBytes);
    if (ns < 2) ns = 2;
    const size_t smem = ns * (size_t)kTileBytes + fixed;
    cudaFuncSetAttribute(solve_umma_kernel<PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ntask * CR, (nrhs + PG - 1) / PG, 1);
    cfg.blockDim = dim3(32 * (5 + kIssuers), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CR;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, solve_umma_kernel<PG>, tasks, subs, nrhs, CR, afac, afac_off, Pv, inva,
                       buf, rstride, ns, ds);
}

bool umma_supported(int nblk_max) { return umma_tiles(nblk_max) <= 2; }

void launch_solve_umma(const Task* tasks, int ntask, const SubDesc* subs, int nblk_max, int nrhs,
                       int panel, const float* afac, const int64_t* afac_off,
                       const cplx<float>* Pv, const cplx<float>* inva, cplx<float>* buf,
                       int64_t rstride, DevStatus ds, cudaStream_t st) {
    if (ntask == 0) return;
    const int CR = umma_tiles(nblk_max);  // cluster of one CTA per 128-row tile
    int nkc = 0;
    umma_line_bytes(nblk_max, CR, &nkc);
#define HELM_UMMA(PG_) \
    launch_pg<PG_>(tasks, ntask, subs, CR, nkc, nrhs, afac, afac_off, Pv, inva, buf, rstride, ds, st)
    if (panel >= 32) HELM_UMMA(32); else if (panel >= 16) HELM_UMMA(16); else HELM_UMMA(8);
#undef HELM_UMMA
}

}  // namespace helm
