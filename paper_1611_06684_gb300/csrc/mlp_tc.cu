// Fused proposal MLP on the fifth-generation tensor cores (tcgen05, sm_103a).
//
//   Z = relu(relu(X W1^T + rowbias) W2^T + b2) W3^T + b3
//
// for rows r = b * C + c of the learned sweep, X [R][Kx] bf16 (the centred
// field features; the block's pair couplings enter as the per-block first
// layer bias), W1 [H][Kx], W2 [H][H], W3 [O][H] bf16, float32 accumulation,
// hidden activations rounded to bf16 between layers (as the GEMM path does).
//
// One CTA of 256 threads owns a 128-row tile at a time (persistent over
// tiles, two CTAs per SM, so one CTA's epilogue overlaps the other's MMAs).
// Two warps share each 32-lane quarter of tensor memory and split the columns
// in the epilogues.  Operands live in shared memory in the K-major,
// 128-byte-swizzled layout the tensor core reads; accumulators live in tensor
// memory (256 columns per CTA) and are read back with tcgen05.ld by the
// thread that owns the row.  The hidden activations never leave the SM: the
// activation tile doubles as the X tile of GEMM 1 and is overwritten by each
// epilogue once the GEMM that read it has completed.  Weights are streamed
// through a two-slot ring of 16 KB chunks (one 64-wide K block of up to 128
// weight rows) by bulk copies from pre-swizzled images in global memory, so a
// plain byte copy lands them in the layout the tensor core expects; the copy
// of the next chunk is in flight while the MMAs of the current one run.  Thread 0 issues the
// copies and the MMAs; every wait is bounded and on a timeout the kernel
// records an error, drains what it issued and frees its tensor memory; if a
// drain wait also gives up it sets a second error bit (the host then refuses
// further learned sweeps on the handle, which must be recreated).
#include "common.cuh"

#include <cuda_bf16.h>

namespace mrfk {

using bf16 = __nv_bfloat16;

namespace tc {
constexpr int TILE_M = 128;              // rows per tile = TMEM lanes
constexpr int THREADS = 256;
constexpr int CHUNK_ROWS = 128;          // weight rows per chunk (N of one MMA)
constexpr int CHUNK_BYTES = CHUNK_ROWS * 128;
constexpr int NSLOT = 2;
constexpr uint32_t TMEM_COLS = 256;
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;   // a wait gives up after one second
}  // namespace tc

// Byte offset of element (row, col) in a K-major, 128-byte-swizzled image of
// a matrix with `rows` rows (rows % 8 == 0): 64-column K block kb starts at
// kb * rows * 128; row r of a block at (r / 8) * 1024 + (r % 8) * 128; the
// 16-byte chunk j = (col % 64) / 8 of a row sits at chunk position j ^ (r % 8).
__host__ __device__ inline uint32_t sw128_offset(int row, int col, int rows) {
    const int kb = col >> 6, c = col & 63;
    return (uint32_t)kb * (uint32_t)rows * 128u + (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u +
           (uint32_t)(((c >> 3) ^ (row & 7)) << 4) + (uint32_t)((c & 7) << 1);
}

// dst = swizzled image of src [N][K] (row-major bf16), K padded with zeros to Kp.
__global__ void k_sw128_image(const bf16* __restrict__ src, int N, int K, int Kp, bf16* __restrict__ dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * Kp) return;
    const int n = (int)(i / Kp), k = (int)(i - (int64_t)n * Kp);
    const bf16 v = k < K ? src[(int64_t)n * K + k] : __float2bfloat16(0.0f);
    *reinterpret_cast<bf16*>(reinterpret_cast<char*>(dst) + sw128_offset(n, k, N)) = v;
}

// ---------------------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the completion of the phase with the given parity; false after
// WAIT_LIMIT_NS of global time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t start = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - start > tc::WAIT_LIMIT_NS) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: bf16 A and B (K-major), float32 D, M x N.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive float32 columns of this thread's TMEM lane.  The load and
// its wait are one asm statement, so no use of the registers can be scheduled
// before the data has arrived.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------- kernel

struct MlpTc {
    const bf16* X;            // [R][Kx]
    int64_t R;
    int Kx, Kxp, H, O, C;     // Kxp = Kx rounded up to 64
    FastDiv fdC;              // rows per block bias
    const float* rowbias;     // [R / C][H]
    const float* b2;          // [H]
    const float* b3;          // [O]
    const uint8_t* w1;        // swizzled images: [H] x Kxp, [H] x H, [O] x H
    const uint8_t* w2;
    const uint8_t* w3;
    float* Z;                 // [R][O]
    unsigned* err;            // bit 0: a wait timed out
    int skip_first_commit;    // test hook: GEMM 1 of the first tile never signals completion
};

// Chunk q of a tile's weight sequence: GEMM g (0..2), K block kb, row half nh.
struct Chunk {
    int gemm, kb, nh, rows;
    const uint8_t* src;
};

__device__ __forceinline__ Chunk chunk_of(const MlpTc& p, int q) {
    const int h_halves = (p.H + tc::CHUNK_ROWS - 1) / tc::CHUNK_ROWS;
    const int o_halves = (p.O + tc::CHUNK_ROWS - 1) / tc::CHUNK_ROWS;
    const int n1 = (p.Kxp / 64) * h_halves, n2 = (p.H / 64) * h_halves;
    Chunk c;
    int N;
    const uint8_t* img;
    int halves;
    if (q < n1) { c.gemm = 0; N = p.H; img = p.w1; halves = h_halves; }
    else if (q < n1 + n2) { c.gemm = 1; q -= n1; N = p.H; img = p.w2; halves = h_halves; }
    else { c.gemm = 2; q -= n1 + n2; N = p.O; img = p.w3; halves = o_halves; }
    c.kb = q / halves;
    c.nh = q - c.kb * halves;
    c.rows = min(tc::CHUNK_ROWS, N - c.nh * tc::CHUNK_ROWS);
    c.src = img + (int64_t)c.kb * N * 128 + (int64_t)c.nh * tc::CHUNK_BYTES;
    return c;
}

__global__ void __launch_bounds__(tc::THREADS, 2) k_mlp_tc(const MlpTc p) {
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned operand area: activation tile, then the weight ring
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int act_cols = p.Kxp > p.H ? p.Kxp : p.H;
    uint8_t* act = base;                                            // 128 rows x act_cols bf16, swizzled
    uint8_t* ring = act + tc::TILE_M * act_cols * 2;                // NSLOT x 16 KB
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + tc::NSLOT * tc::CHUNK_BYTES);
    // bars[0..NSLOT): full, [NSLOT..2 NSLOT): empty, [2 NSLOT]: done, [2 NSLOT + 1]: drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * tc::NSLOT + 2);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + tc::NSLOT);
    const uint32_t done = smem_u32(bars + 2 * tc::NSLOT), drain = smem_u32(bars + 2 * tc::NSLOT + 1);

    if (tid == 0) {
        for (int i = 0; i < 2 * tc::NSLOT + 2; ++i) mbar_init(smem_u32(bars + i), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(tc::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int h_halves = (p.H + tc::CHUNK_ROWS - 1) / tc::CHUNK_ROWS;
    const int o_halves = (p.O + tc::CHUNK_ROWS - 1) / tc::CHUNK_ROWS;
    const int per_gemm[3] = {(p.Kxp / 64) * h_halves, (p.H / 64) * h_halves, (p.H / 64) * o_halves};
    const int per_tile = per_gemm[0] + per_gemm[1] + per_gemm[2];
    const int64_t n_tiles = (p.R + tc::TILE_M - 1) / tc::TILE_M;
    const int64_t my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = my_tiles * per_tile;                      // chunks this CTA consumes

    // thread 0: chunk producer and MMA issuer; q_load / q_mma count chunks
    int64_t q_load = 0, q_mma = 0;
    uint32_t done_phase = 0;
    bool ok = true;
    // issue copies while the ring has room: up to NSLOT - 1 chunks ahead of the
    // MMAs, so refilling a slot only waits for MMAs two chunks back or more
    auto top_up = [&]() {                                          // thread 0 only
        while (ok && q_load < total && q_load < q_mma + tc::NSLOT - 1) {
            const int slot = (int)(q_load % tc::NSLOT);
            const int64_t use = q_load / tc::NSLOT;
            if (use > 0 && !mbar_wait(empty0 + 8 * slot, (uint32_t)((use - 1) & 1))) { ok = false; return; }
            const Chunk ch = chunk_of(p, (int)(q_load % per_tile));
            const uint32_t bytes = (uint32_t)ch.rows * 128u;
            mbar_expect_tx(full0 + 8 * slot, bytes);
            bulk_g2s(smem_u32(ring + slot * tc::CHUNK_BYTES), ch.src, bytes, full0 + 8 * slot);
            ++q_load;
        }
    };
    // MMAs of every chunk of GEMM g of the current tile, then commit to `done`;
    // the ring is topped up after each chunk's MMAs are queued (copies of the
    // next GEMM's chunks land during the epilogue)
    auto run_gemm = [&](int g) {                                   // thread 0 only
        for (int i = 0; i < per_gemm[g] && ok; ++i) {
            top_up();
            if (!ok) break;
            const int slot = (int)(q_mma % tc::NSLOT);
            if (!mbar_wait(full0 + 8 * slot, (uint32_t)((q_mma / tc::NSLOT) & 1))) { ok = false; break; }
            tc_fence_after();
            const Chunk ch = chunk_of(p, (int)(q_mma % per_tile));
            const uint32_t idesc = f16_idesc(tc::TILE_M, ch.rows);
            const uint32_t a0 = smem_u32(act) + (uint32_t)ch.kb * (tc::TILE_M * 128u);
            const uint32_t b0 = smem_u32(ring + slot * tc::CHUNK_BYTES);
            const uint32_t d = tmem + (uint32_t)(ch.nh * tc::CHUNK_ROWS);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_bf16(d, sw128_desc(a0 + 32u * k), sw128_desc(b0 + 32u * k), idesc, (ch.kb > 0 || k > 0) ? 1u : 0u);
            mma_commit(empty0 + 8 * slot);                         // slot free once these MMAs finish
            ++q_mma;
            top_up();
        }
        if (ok && !(p.skip_first_commit && g == 0 && q_mma == per_gemm[0])) mma_commit(done);
    };

    const int row = tid & (tc::TILE_M - 1);                        // tile row = TMEM lane
    const int half = tid >> 7;                                     // which 32-column chunks this thread takes
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t r = t * tc::TILE_M + row;
        // X tile -> activation area (K-major swizzled), zero rows past R and columns past Kx
        {
            const uint4* xr = reinterpret_cast<const uint4*>(p.X + (r < p.R ? r : 0) * (int64_t)p.Kx);
            for (int c8 = half; c8 < p.Kxp / 8; c8 += 2) {
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (r < p.R && c8 * 8 < p.Kx) v = __ldg(xr + c8);
                *reinterpret_cast<uint4*>(act + sw128_offset(row, c8 * 8, tc::TILE_M)) = v;
            }
        }
        proxy_fence_smem();
        tc_fence_before();
        if (__syncthreads_or(!ok)) break;
        for (int g = 0; g < 3; ++g) {
            if (tid == 0) {
                tc_fence_after();
                run_gemm(g);
            }
            // accumulator ready (bounded wait by every thread)
            if (__syncthreads_or(tid == 0 && !ok)) { ok = false; break; }
            const bool ready = mbar_wait(done, done_phase);
            done_phase ^= 1u;
            if (__syncthreads_or(!ready)) { ok = false; break; }
            tc_fence_after();
            const int N = g < 2 ? p.H : p.O;
            const float* bias = g == 1 ? p.b2 : p.b3;
            if (g == 0) bias = p.rowbias + (int64_t)p.fdC.div((uint32_t)(r < p.R ? r : p.R - 1)) * p.H;
            for (int c0 = 32 * half; c0 < N; c0 += 64) {
                float v[32];
                tmem_ld32(lane_addr + (uint32_t)c0, v);
                const float4* b4 = reinterpret_cast<const float4*>(bias + c0);
                if (g < 2) {
                    uint32_t packed[16];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 bq = __ldg(b4 + q);
                        __nv_bfloat162 lo = __floats2bfloat162_rn(fmaxf(v[4 * q] + bq.x, 0.0f), fmaxf(v[4 * q + 1] + bq.y, 0.0f));
                        __nv_bfloat162 hi = __floats2bfloat162_rn(fmaxf(v[4 * q + 2] + bq.z, 0.0f), fmaxf(v[4 * q + 3] + bq.w, 0.0f));
                        packed[2 * q] = *reinterpret_cast<uint32_t*>(&lo);
                        packed[2 * q + 1] = *reinterpret_cast<uint32_t*>(&hi);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<uint4*>(act + sw128_offset(row, c0 + 8 * q, tc::TILE_M)) =
                            make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
                } else if (r < p.R) {
                    float4* zr = reinterpret_cast<float4*>(p.Z + r * (int64_t)p.O + c0);
                    const int nv = min(32, N - c0) / 4;
                    for (int q = 0; q < nv; ++q) {
                        const float4 bq = __ldg(b4 + q);
                        zr[q] = make_float4(v[4 * q] + bq.x, v[4 * q + 1] + bq.y, v[4 * q + 2] + bq.z, v[4 * q + 3] + bq.w);
                    }
                }
            }
            proxy_fence_smem();
            tc_fence_before();
            __syncthreads();
        }
        if (!ok) break;
    }

    // shutdown: on a timeout, record it and let everything issued finish
    // (bounded) before the tensor memory is released
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicOr(p.err, 1u);
            mma_commit(drain);                                     // completes after all issued MMAs
            bool drained = mbar_wait(drain, 0);
            for (int64_t q = q_mma; q < q_load; ++q)                // copies issued but not consumed
                drained &= mbar_wait(full0 + 8 * (int)(q % tc::NSLOT), (uint32_t)((q / tc::NSLOT) & 1));
            if (!drained) atomicOr(p.err, 2u);                    // work may still be in flight: handle unusable
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc::TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------------- resident-weight form

// When W1, W2 and W3 fit in shared memory together (<= 200 KB of bf16) they are
// copied in once per CTA and stay there; the activations then live in tensor
// memory instead of shared memory: each GEMM's A operand (X, then H1, then H2,
// 128 rows x K bf16, two values per 32-bit column, row = lane) is written by
// the epilogue with tcgen05.st next to the accumulator (columns [0, 256) hold
// the accumulator, [256, 384) the A operand).  No weight bytes move per tile.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
          "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
          "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D (tmem) += A (tmem, K-packed) x B^T (shared, K-major swizzled)
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(d_tmem), "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

namespace tcr {
constexpr int THREADS = 512;               // four warps per 32-lane quarter of tensor memory
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACOL = 256;            // first column of the A operand
constexpr int MAX_SMEM = 220 * 1024;      // weights + X staging
}  // namespace tcr

// Stage the X rows of tile t (row-major, Kxp bf16 per row, zero padded) with
// cp.async; every thread issues its share of the 16-byte pieces.
__device__ __forceinline__ void stage_x(const MlpTc& p, int64_t t, uint8_t* stage) {
    const int pieces_per_row = p.Kxp / 8;
    const int pieces = 128 * pieces_per_row;
    for (int i = threadIdx.x; i < pieces; i += blockDim.x) {
        const int rr = i / pieces_per_row, c8 = i - rr * pieces_per_row;
        const int64_t r = t * 128 + rr;
        const bool in = r < p.R && c8 * 8 < p.Kx;
        const bf16* src = p.X + (in ? r * (int64_t)p.Kx + c8 * 8 : 0);
        cp_async16_zfill(smem_u32(stage + (size_t)i * 16), src, in ? 16u : 0u);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(tcr::THREADS, 1) k_mlp_tc_resident(const MlpTc p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int64_t w1b = 2 * (int64_t)p.H * p.Kxp, w2b = 2 * (int64_t)p.H * p.H, w3b = 2 * (int64_t)p.O * p.H;
    uint8_t* w1s = base;
    uint8_t* w2s = w1s + w1b;
    uint8_t* w3s = w2s + w2b;
    uint8_t* stage = w3s + ((w3b + 15) & ~(int64_t)15);             // X rows of the next tile
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage + 128 * (int64_t)p.Kxp * 2);    // [0]: weights, [1]: done, [2]: drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t wbar = smem_u32(bars), done = smem_u32(bars + 1), drain = smem_u32(bars + 2);
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(smem_u32(bars + i), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(tcr::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // weights: one barrier, copies of at most 32 KB each
    if (tid == 0) {
        mbar_expect_tx(wbar, (uint32_t)(w1b + w2b + w3b));
        const uint8_t* src[3] = {p.w1, p.w2, p.w3};
        uint8_t* dst[3] = {w1s, w2s, w3s};
        const int64_t len[3] = {w1b, w2b, w3b};
        for (int k = 0; k < 3; ++k)
            for (int64_t o = 0; o < len[k]; o += 32768)
                bulk_g2s(smem_u32(dst[k] + o), src[k] + o, (uint32_t)std::min<int64_t>(32768, len[k] - o), wbar);
    }
    const int64_t n_tiles = (p.R + 127) / 128;
    if (blockIdx.x < n_tiles) stage_x(p, blockIdx.x, stage);
    bool ok = !__syncthreads_or(!mbar_wait(wbar, 0));              // the same verdict in every thread
    const int row = tid & 127, quarter = tid >> 7;
    const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t acc_addr = tmem + lane, a_addr = tmem + lane + tcr::ACOL;
    uint32_t done_phase = 0;
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int64_t r = t * 128 + row;
        // staged X rows -> A operand: 16 packed columns (32 bf16) per step, quarters alternate
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        for (int c0 = 16 * quarter; c0 < p.Kxp / 2; c0 += 64) {
            const uint4* src = reinterpret_cast<const uint4*>(stage + (size_t)row * p.Kxp * 2 + (size_t)c0 * 4);
            uint32_t w[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 v = src[q];
                w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
            }
            tmem_st16(a_addr + (uint32_t)c0, w);
        }
        tmem_st_wait();
        __syncthreads();                                           // staging read by all before it is refilled
        if (t + gridDim.x < n_tiles) stage_x(p, t + gridDim.x, stage);
        for (int g = 0; g < 3 && ok; ++g) {
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const int K = g == 0 ? p.Kxp : p.H, N = g < 2 ? p.H : p.O;
                const uint8_t* ws = g == 0 ? w1s : (g == 1 ? w2s : w3s);
                const uint32_t idesc = f16_idesc(128, N);
                for (int j = 0; j < K / 16; ++j) {
                    const uint32_t b = smem_u32(ws) + (uint32_t)(j >> 2) * (uint32_t)N * 128u + 32u * (uint32_t)(j & 3);
                    mma_bf16_ts(tmem, tmem + tcr::ACOL + 8u * (uint32_t)j, sw128_desc(b), idesc, j > 0 ? 1u : 0u);
                }
                if (!(p.skip_first_commit && g == 0 && t == blockIdx.x)) mma_commit(done);
            }
            const bool ready = mbar_wait(done, done_phase);
            done_phase ^= 1u;
            if (__syncthreads_or(!ready)) { ok = false; break; }
            tc_fence_after();
            const int N = g < 2 ? p.H : p.O;
            const float* bias = g == 1 ? p.b2 : p.b3;
            if (g == 0) bias = p.rowbias + (int64_t)p.fdC.div((uint32_t)(r < p.R ? r : p.R - 1)) * p.H;
            // 32 accumulator columns (16 packed A columns) per step, quarters alternate
            for (int c0 = 32 * quarter; c0 < N; c0 += 128) {
                float v[32];
                tmem_ld32(acc_addr + (uint32_t)c0, v);
                const float4* b4 = reinterpret_cast<const float4*>(bias + c0);
                if (g < 2) {
                    uint32_t packed[16];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 bq = __ldg(b4 + q);
                        __nv_bfloat162 lo = __floats2bfloat162_rn(fmaxf(v[4 * q] + bq.x, 0.0f), fmaxf(v[4 * q + 1] + bq.y, 0.0f));
                        __nv_bfloat162 hi = __floats2bfloat162_rn(fmaxf(v[4 * q + 2] + bq.z, 0.0f), fmaxf(v[4 * q + 3] + bq.w, 0.0f));
                        packed[2 * q] = *reinterpret_cast<uint32_t*>(&lo);
                        packed[2 * q + 1] = *reinterpret_cast<uint32_t*>(&hi);
                    }
                    tmem_st16(a_addr + (uint32_t)(c0 / 2), packed);
                } else if (r < p.R) {
                    float4* zr = reinterpret_cast<float4*>(p.Z + r * (int64_t)p.O + c0);
                    const int nv = min(32, N - c0) / 4;
                    for (int q = 0; q < nv; ++q) {
                        const float4 bq = __ldg(b4 + q);
                        zr[q] = make_float4(v[4 * q] + bq.x, v[4 * q + 1] + bq.y, v[4 * q + 2] + bq.z, v[4 * q + 3] + bq.w);
                    }
                }
            }
            if (g < 2) tmem_st_wait();
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicOr(p.err, 1u);
            mma_commit(drain);
            bool drained = mbar_wait(drain, 0);
            drained &= mbar_wait(wbar, 0);
            if (!drained) atomicOr(p.err, 2u);                    // work may still be in flight: handle unusable
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcr::TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------------- host side

bool mlp_tc_supported(const LearnedArgs& a) {
    return a.wimg && a.H % 64 == 0 && a.H <= 256 && a.O % 16 == 0 && a.O <= 256 && a.Kx % 8 == 0 && a.Kx <= 256;
}

static int64_t kxp_of(const LearnedArgs& a) { return (a.Kx + 63) / 64 * 64; }

int64_t mlp_tc_image_bytes(int H, int O, int Kx) {
    const int64_t kxp = (Kx + 63) / 64 * 64;
    return 2 * ((int64_t)H * kxp + (int64_t)H * H + (int64_t)O * H);
}

cudaError_t launch_mlp_images(const LearnedArgs& a, cudaStream_t s) {
    if (!mlp_tc_supported(a)) return cudaSuccess;
    const int64_t kxp = kxp_of(a);
    bf16* w1 = reinterpret_cast<bf16*>(a.wimg);
    bf16* w2 = w1 + (int64_t)a.H * kxp;
    bf16* w3 = w2 + (int64_t)a.H * a.H;
    const int64_t n1 = (int64_t)a.H * kxp, n2 = (int64_t)a.H * a.H, n3 = (int64_t)a.O * a.H;
    k_sw128_image<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(a.W1xb, a.H, a.Kx, (int)kxp, w1);
    k_sw128_image<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(a.W2b, a.H, a.H, a.H, w2);
    k_sw128_image<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(a.W3b, a.O, a.H, a.H, w3);
    return cudaGetLastError();
}

cudaError_t launch_learned_mlp_tc(const LearnedArgs& a, cudaStream_t s) {
    MlpTc p;
    p.X = a.X;
    p.R = (int64_t)a.nb * a.C;
    p.Kx = a.Kx;
    p.Kxp = (int)kxp_of(a);
    p.H = a.H;
    p.O = a.O;
    p.C = a.C;
    p.fdC = FastDiv::make((uint32_t)a.C);
    p.rowbias = a.rowbias;
    p.b2 = a.b2;
    p.b3 = a.b3;
    p.w1 = a.wimg;
    p.w2 = p.w1 + 2 * (int64_t)a.H * p.Kxp;
    p.w3 = p.w2 + 2 * (int64_t)a.H * a.H;
    p.Z = a.Zm;
    p.err = a.tc_err;
    p.skip_first_commit = a.tc_inject_timeout;
    if (p.R == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t n_tiles = (p.R + tc::TILE_M - 1) / tc::TILE_M;
    const int64_t wbytes = 2 * ((int64_t)p.H * p.Kxp + (int64_t)p.H * p.H + (int64_t)p.O * p.H);
    const int64_t resident_bytes = 1024 + wbytes + 16 + 128 * (int64_t)p.Kxp * 2 + 64;
    if (resident_bytes <= tcr::MAX_SMEM && p.Kxp <= 256 && p.H <= 256) {
        // at least 120 KB: one CTA (512 TMEM columns) per SM
        const size_t smem = std::max<size_t>(120 * 1024, (size_t)resident_bytes);
        static int attr_r = 0;
        if ((int)smem > attr_r) {
            e = cudaFuncSetAttribute(k_mlp_tc_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_r = (int)smem;
        }
        k_mlp_tc_resident<<<(unsigned)std::min<int64_t>(n_tiles, sms), tcr::THREADS, smem, s>>>(p);
        return cudaGetLastError();
    }
    const int act_cols = p.Kxp > p.H ? p.Kxp : p.H;
    // at least 80 KB, so that no more than two CTAs (2 x 256 TMEM columns) share an SM
    const size_t smem = std::max<size_t>(80 * 1024,
                                         1024 + (size_t)tc::TILE_M * act_cols * 2 + (size_t)tc::NSLOT * tc::CHUNK_BYTES + 256);
    static int attr_set = 0;                     // largest dynamic shared memory configured so far
    if ((int)smem > attr_set) {
        e = cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = (int)smem;
    }
    const unsigned grid = (unsigned)std::min<int64_t>(n_tiles, 2 * (int64_t)sms);
    k_mlp_tc<<<grid, tc::THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace mrfk
