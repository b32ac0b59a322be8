// rtcg_ptx.cuh -- PTX wrappers shared by the run-time generated tcgen05 kernels
// (the filter-bank correlation of rtcg_tc.cuh and the nearest-neighbour distance
// kernel of rtcg_nn.cuh): shared-memory addresses, mbarriers with time-bounded
// waits, 1D bulk copies, tiled bulk stores, tcgen05.mma / commit / ld (one CTA,
// or a CTA pair with cta_group::2), cluster barriers and remote arrivals, BF16
// packing.  Embedded as a
// string and placed after the kernel's parameter block in every generated
// source; self-contained (no system headers).  A bounded wait takes any
// parameter block with `wait_ns` (the bound) and `err` (the host-mapped error
// word): on expiry it records the caller's code there and raises the CTA's
// abort flag.

typedef unsigned int fbc_u32;
typedef unsigned long long fbc_u64;
typedef unsigned char fbc_u8;

extern __shared__ __align__(1024) fbc_u8 fbc_tc_smem[];

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ fbc_u32 fbc_smem_addr(const void* p) {
    fbc_u32 r;
    asm("{\n .reg .u64 t;\n cvta.to.shared.u64 t, %1;\n cvt.u32.u64 %0, t;\n}\n" : "=r"(r) : "l"(p));
    return r;
}

__device__ __forceinline__ fbc_u64 fbc_globaltimer() {
    fbc_u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void fbc_mbar_init(fbc_u32 bar, fbc_u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool fbc_mbar_try_wait(fbc_u32 bar, fbc_u32 parity) {
    fbc_u32 ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void fbc_mbar_arrive(fbc_u32 bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fbc_mbar_expect_tx(fbc_u32 bar, fbc_u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// 1D bulk copy global -> shared, completion counted on `bar` (bytes % 16 == 0).
__device__ __forceinline__ void fbc_bulk_g2s(fbc_u32 dst, const void* src, fbc_u32 bytes, fbc_u32 bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fbc_tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fbc_tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// K-major, no-swizzle shared-memory matrix descriptor.
__device__ __forceinline__ fbc_u64 fbc_smem_desc(fbc_u32 addr, fbc_u32 lbo, fbc_u32 sbo) {
    return (fbc_u64)((addr & 0x3FFFFu) >> 4) | ((fbc_u64)(lbo >> 4) << 16) | ((fbc_u64)(sbo >> 4) << 32) |
           (1ull << 46);
}

// CG = 1: one CTA, M = 128.  CG = 2: issued by the even CTA of a pair for both
// (M = 256: rows 0..127 from the even CTA's A, 128..255 from the odd CTA's, at the
// same shared-memory offsets; B columns 0..N/2-1 from the even CTA, the rest
// from the odd one; each CTA's TMEM receives its own 128 rows).  Every tcgen05
// instruction of a kernel uses the same CG.
template <int CG = 1>
__device__ __forceinline__ void fbc_umma(fbc_u32 d_tmem, fbc_u64 a, fbc_u64 b, fbc_u32 idesc, fbc_u32 accumulate) {
    if constexpr (CG == 2)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Arrive on the mbarrier at shared::cluster address `bar` (this CTA's, or with
// CG = 2 one of the peer's, from fbc_mapa) once the MMAs issued so far are done.
template <int CG = 1>
__device__ __forceinline__ void fbc_umma_commit(fbc_u32 bar) {
    if constexpr (CG == 2)
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
    else
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
}

// ---------------------------------------------------------------- clusters
__device__ __forceinline__ fbc_u32 fbc_cluster_rank() {
    fbc_u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of every CTA of the cluster (release / acquire at cluster scope).
__device__ __forceinline__ void fbc_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The shared::cluster address of shared-memory address `addr` in CTA `rank` of the cluster.
__device__ __forceinline__ fbc_u32 fbc_mapa(fbc_u32 addr, fbc_u32 rank) {
    fbc_u32 r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Arrive on an mbarrier of another CTA of the cluster.  The default (CTA-scope)
// release: what the arrival publishes lives in shared memory and TMEM, which
// the peer reaches directly.  With a cluster-scope release, which also orders
// global memory across SMs, a relay forwarding every B stage took about 0.6 us
// per stage.
__device__ __forceinline__ void fbc_mbar_arrive_remote(fbc_u32 cluster_addr) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// tcgen05.ld 16x256b.x8 -- 16 TMEM lanes x 64 columns: registers 4g, 4g+1 hold
// columns 8g + 2*(lane%4) + {0,1} of lane lane/4, registers 4g+2, 4g+3 the same
// columns of lane 8 + lane/4.
// Issued without its wait: several loads can be in flight before one
// fbc_tmem_ld_wait(); fbc_reg_fence() then orders every use of the registers
// after that wait.
__device__ __forceinline__ void fbc_tmem_ld16x256b_x8_async(fbc_u32 taddr, fbc_u32 (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// tcgen05.ld 32x32b.x32 -- 32 TMEM lanes x 32 columns: register j holds column
// j of lane `lane` (one accumulator row per thread).  Issued without its wait.
__device__ __forceinline__ void fbc_tmem_ld32x32b_x32_async(fbc_u32 taddr, fbc_u32 (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void fbc_tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void fbc_reg_fence(fbc_u32 (&r)[32]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        asm volatile("" : "+r"(r[8 * q]), "+r"(r[8 * q + 1]), "+r"(r[8 * q + 2]), "+r"(r[8 * q + 3]),
                     "+r"(r[8 * q + 4]), "+r"(r[8 * q + 5]), "+r"(r[8 * q + 6]), "+r"(r[8 * q + 7]));
}

// Streaming 8-byte store.
__device__ __forceinline__ void fbc_st_cs_f2(float* p, float a, float b) {
    asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

// 16-byte shared store.
__device__ __forceinline__ void fbc_st_shared_v4(fbc_u32 addr, fbc_u32 a, fbc_u32 b, fbc_u32 c, fbc_u32 d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ uint4 fbc_ld_shared_v4(fbc_u32 addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
                 : "memory");
    return v;
}

// Streaming 16-byte store.
__device__ __forceinline__ void fbc_st_cs_v4(float* p, uint4 v) {
    asm volatile("st.global.cs.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// Make this thread's shared-memory writes visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void fbc_fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Tiled bulk store shared -> global of one box of a 3D tensor map (coordinates
// innermost first, all >= 0; elements outside the tensor are not written),
// tracked in this thread's bulk async-group.
__device__ __forceinline__ void fbc_tma_store_3d(const void* tmap, fbc_u32 src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(tmap),
                 "r"(src), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

__device__ __forceinline__ void fbc_bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until at most N of this thread's bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void fbc_bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until every bulk group of this thread has completed its writes.
__device__ __forceinline__ void fbc_bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Two FP32 values -> two BF16 (round to nearest even), packed low = a, high = b.
__device__ __forceinline__ fbc_u32 fbc_pack_bf16x2(float a, float b) {
    fbc_u32 r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

// hi = bf16_rn(v), lo = bf16_rn(v - hi) for 8 values; v - hi is exact in FP32.
template <int SPLIT>
__device__ __forceinline__ void fbc_split8(const float (&v)[8], uint4* hi_out, uint4* lo_out) {
    fbc_u32 h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h[k] = fbc_pack_bf16x2(v[2 * k], v[2 * k + 1]);
        if (SPLIT) {
            const float h0 = __uint_as_float(h[k] << 16);
            const float h1 = __uint_as_float(h[k] & 0xFFFF0000u);
            l[k] = fbc_pack_bf16x2(v[2 * k] - h0, v[2 * k + 1] - h1);
        }
    }
    *hi_out = make_uint4(h[0], h[1], h[2], h[3]);
    if (SPLIT) *lo_out = make_uint4(l[0], l[1], l[2], l[3]);
}

// ---------------------------------------------------------------- bounded waits
template <class Prm>
__device__ __noinline__ bool fbc_wait_slow(fbc_u32 bar, fbc_u32 parity, const Prm& P,
                                           volatile int* abort_flag, int code) {
    const fbc_u64 t0 = fbc_globaltimer();
    for (;;) {
#pragma unroll 1
        for (int k = 0; k < 64; ++k)
            if (fbc_mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (fbc_globaltimer() - t0 > P.wait_ns) {
            *abort_flag = 1;
            *(volatile int*)P.err = code;
            __threadfence_system();
            return false;
        }
    }
}

template <class Prm>
__device__ __forceinline__ bool fbc_wait(fbc_u32 bar, fbc_u32 parity, const Prm& P,
                                         volatile int* abort_flag, int code) {
    if (fbc_mbar_try_wait(bar, parity)) return true;
    return fbc_wait_slow(bar, parity, P, abort_flag, code);
}

// Drain wait after an abort: bounded, ignores the abort flag.
template <class Prm>
__device__ __noinline__ void fbc_wait_drain(fbc_u32 bar, fbc_u32 parity, const Prm& P) {
    const fbc_u64 t0 = fbc_globaltimer();
    while (!fbc_mbar_try_wait(bar, parity))
        if (fbc_globaltimer() - t0 > P.wait_ns) return;
}

