// CUDA kernels of Cosm for sm_103a.
//
// One CTA owns a tile of K replicas and keeps all their phases resident in
// shared memory, interleaved [slot][replica], for a whole segment of sweeps.
// A sub-sweep (one colour, a matching: Section II-C) maps edges to threads;
// no vertex repeats inside a colour, so the read-modify-write of both
// endpoints needs no atomics, and one __syncthreads separates colours.
// The DWT (Section II-D), the step schedule and the bisector readout with
// exact integer cuts (Alg. 1) are fused into the same kernel.
//
// Phase representation: turns, held as the representative g in [-1/2, 1/2]
// (g = x for x < 1/2, g = x - 1 otherwise). Every wrap is then
// g - rint(g), which is exact in binary32; rint uses the 1.5 * 2^23 addend
// (valid for |g| < 2^22), so the hot loop is plain FP32 adds.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "../../include/cosm.h"
#include "cosm_internal.h"

namespace cosm {

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll 1
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Top 24 bits of a word as a turn in [0,1), mapped to its representative in
// [-1/2, 1/2); exact in FP32.
__device__ __forceinline__ float u24_centered(uint32_t word)
{
    const float x = (float)(word >> 8) * 0x1p-24f;
    return x >= 0.5f ? x - 1.0f : x;
}

// DWT reference angle for (seed, replica, sweep): counter (s, r, 0, 1),
// word 0; the top bit of word 1 is the drawn twist direction (set: -1).
__device__ __forceinline__ float dwt_theta(uint64_t seed, uint32_t replica, int64_t sweep, bool *neg = nullptr)
{
    uint32_t c[4] = {(uint32_t)sweep, replica, 0u, 1u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    if (neg) *neg = (c[1] >> 31) != 0;
    return (float)(c[0] >> 8) * 0x1p-24f;  // [0, 1), exact
}

// ---------------------------------------------------------------- arithmetic
__device__ __forceinline__ float rint_fast(float v)
{
    return __fadd_rn(__fadd_rn(v, 12582912.0f), -12582912.0f);
}
__device__ __forceinline__ float wrap_c(float v) { return __fadd_rn(v, -rint_fast(v)); }

// q = floor(x 2^32) mod 2^32 of the turn x represented by g (exact).
__device__ __forceinline__ uint32_t phase_q(float g)
{
    return (uint32_t)(unsigned long long)__float2ll_rd(g * 4294967296.0f);
}

// ---------------------------------------------------------------- checked build
// With COSM_CHECKS defined (the checked library, a stand-in for a memory
// checker), device code validates the indices it is given: an edge record's
// two slots must lie below n and a lattice layout must tile its slots; a
// failed check sets bit 2 of the handle's error word (cosm_sync then reports
// COSM_ERR_CHECK) and the access goes to slot 0 instead. The normal build
// compiles the checks away.
__device__ __forceinline__ uint32_t checked_rec(const InstView &a, uint32_t rec)
{
#ifdef COSM_CHECKS
    if ((rec & 0xFFFFu) >= (uint32_t)a.n || (rec >> 16) >= (uint32_t)a.n) {
        if (a.check) atomicOr(a.check, 2);
        return 0u;
    }
#else
    (void)a;
#endif
    return rec;
}
__device__ __forceinline__ uint32_t load_rec(const InstView &a, int e) { return checked_rec(a, __ldg(a.ij + e)); }
// A record of a.ijs ([w = -1] | slot(src) << 1 | slot(dst) << 16).
__device__ __forceinline__ uint32_t load_rec_sgn(const InstView &a, int e)
{
    const uint32_t rec = __ldg(a.ijs + e);
#ifdef COSM_CHECKS
    if (((rec & 0xFFFFu) >> 1) >= (uint32_t)a.n || (rec >> 16) >= (uint32_t)a.n) {
        if (a.check) atomicOr(a.check, 2);
        return 0u;
    }
#endif
    return rec;
}

// ---------------------------------------------------------------- storage
template <int K>
__device__ __forceinline__ void ldk(const float *p, float (&x)[K])
{
    if constexpr (K == 1) {
        x[0] = p[0];
    } else if constexpr (K == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        x[0] = v.x; x[1] = v.y;
    } else {
        static_assert(K == 4, "K");
        const float4 v = *reinterpret_cast<const float4 *>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
}
template <int K>
__device__ __forceinline__ void stk(float *p, const float (&x)[K])
{
    if constexpr (K == 1) {
        p[0] = x[0];
    } else if constexpr (K == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
    } else {
        *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
}
// Two 16-bit floats (binary16 or bfloat16) packed in a 32-bit word, to and
// from two binary32 values (round to nearest even on the way in).
template <typename H>
__device__ __forceinline__ float2 h2_to_f2(uint32_t u)
{
    if constexpr (std::is_same<H, __half>::value) {
        __half2 h;
        memcpy(&h, &u, 4);
        return __half22float2(h);
    } else {
        __nv_bfloat162 h;
        memcpy(&h, &u, 4);
        return __bfloat1622float2(h);
    }
}
template <typename H>
__device__ __forceinline__ uint32_t f2_to_h2(float a, float b)
{
    uint32_t u;
    if constexpr (std::is_same<H, __half>::value) {
        const __half2 h = __floats2half2_rn(a, b);
        memcpy(&u, &h, 4);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        memcpy(&u, &h, 4);
    }
    return u;
}
template <typename H, int K>
__device__ __forceinline__ void ldk16(const H *p, float (&x)[K])
{
    if constexpr (K == 2) {
        const float2 f = h2_to_f2<H>(*reinterpret_cast<const uint32_t *>(p));
        x[0] = f.x; x[1] = f.y;
    } else if constexpr (K == 4) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        float2 f = h2_to_f2<H>(u.x); x[0] = f.x; x[1] = f.y;
        f = h2_to_f2<H>(u.y); x[2] = f.x; x[3] = f.y;
    } else {
        static_assert(K == 8, "K");
        const uint4 u = *reinterpret_cast<const uint4 *>(p);
        float2 f = h2_to_f2<H>(u.x); x[0] = f.x; x[1] = f.y;
        f = h2_to_f2<H>(u.y); x[2] = f.x; x[3] = f.y;
        f = h2_to_f2<H>(u.z); x[4] = f.x; x[5] = f.y;
        f = h2_to_f2<H>(u.w); x[6] = f.x; x[7] = f.y;
    }
}
template <typename H, int K>
__device__ __forceinline__ void stk16(H *p, const float (&x)[K])
{
    if constexpr (K == 2) {
        *reinterpret_cast<uint32_t *>(p) = f2_to_h2<H>(x[0], x[1]);
    } else if constexpr (K == 4) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(f2_to_h2<H>(x[0], x[1]), f2_to_h2<H>(x[2], x[3]));
    } else {
        *reinterpret_cast<uint4 *>(p) = make_uint4(f2_to_h2<H>(x[0], x[1]), f2_to_h2<H>(x[2], x[3]),
                                                   f2_to_h2<H>(x[4], x[5]), f2_to_h2<H>(x[6], x[7]));
    }
}
template <int K>
__device__ __forceinline__ void ldk(const __half *p, float (&x)[K]) { ldk16<__half, K>(p, x); }
template <int K>
__device__ __forceinline__ void stk(__half *p, const float (&x)[K]) { stk16<__half, K>(p, x); }
template <int K>
__device__ __forceinline__ void ldk(const __nv_bfloat16 *p, float (&x)[K]) { ldk16<__nv_bfloat16, K>(p, x); }
template <int K>
__device__ __forceinline__ void stk(__nv_bfloat16 *p, const float (&x)[K]) { stk16<__nv_bfloat16, K>(p, x); }

// A binary32 value in a storage type (round to nearest even).
template <typename Store>
__device__ __forceinline__ Store to_store(float v)
{
    if constexpr (std::is_same<Store, __half>::value) return __float2half_rn(v);
    else if constexpr (std::is_same<Store, __nv_bfloat16>::value) return __float2bfloat16_rn(v);
    else return v;
}

// COSM_Q16 phases: integers on the 2^-16-turn grid stored as u16. In
// registers a phase is the 32-bit integer q << 16, so 32-bit wrap-around is
// the modular arithmetic of the circle and needs no wrap step; steps are
// integers on the same grid, so every update is exact.
template <int K>
__device__ __forceinline__ void ldq(const uint16_t *p, uint32_t (&x)[K])
{
    if constexpr (K == 2) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(p);
        x[0] = w << 16; x[1] = w & 0xFFFF0000u;
    } else if constexpr (K == 4) {
        const uint2 w = *reinterpret_cast<const uint2 *>(p);
        x[0] = w.x << 16; x[1] = w.x & 0xFFFF0000u;
        x[2] = w.y << 16; x[3] = w.y & 0xFFFF0000u;
    } else {
        static_assert(K == 8, "K");
        const uint4 w = *reinterpret_cast<const uint4 *>(p);
        x[0] = w.x << 16; x[1] = w.x & 0xFFFF0000u;
        x[2] = w.y << 16; x[3] = w.y & 0xFFFF0000u;
        x[4] = w.z << 16; x[5] = w.z & 0xFFFF0000u;
        x[6] = w.w << 16; x[7] = w.w & 0xFFFF0000u;
    }
}
// low half-word from a's top half, high half-word from b's top half
__device__ __forceinline__ uint32_t pack_q(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x7632); }
template <int K>
__device__ __forceinline__ void stq(uint16_t *p, const uint32_t (&x)[K])
{
    if constexpr (K == 2) {
        *reinterpret_cast<uint32_t *>(p) = pack_q(x[0], x[1]);
    } else if constexpr (K == 4) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(pack_q(x[0], x[1]), pack_q(x[2], x[3]));
    } else {
        *reinterpret_cast<uint4 *>(p) = make_uint4(pack_q(x[0], x[1]), pack_q(x[2], x[3]),
                                                   pack_q(x[4], x[5]), pack_q(x[6], x[7]));
    }
}

// q = floor(x 2^32) mod 2^32 of each of K phases, for any storage type.
template <typename Store, int K>
__device__ __forceinline__ void ld_q32(const Store *p, uint32_t (&q)[K])
{
    if constexpr (std::is_same<Store, uint16_t>::value) {
        ldq<K>(p, q);
    } else {
        float x[K];
        ldk<K>(p, x);
#pragma unroll
        for (int r = 0; r < K; ++r) q[r] = phase_q(x[r]);
    }
}

__host__ __device__ constexpr size_t round16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename Store, int K>
__host__ __device__ constexpr size_t phase_bytes(int n)
{
    return round16((size_t)n * K * sizeof(Store));
}

// Shared layout: phases | NO_SCS accumulators (FP32, n*K) | readout
// difference arrays (int32, K*(P+1)) | per-replica words: DWT offsets,
// twist steps, readout flags, bisector positions, second DWT offsets (5K).
template <typename Store, int K>
__host__ __device__ constexpr size_t smem_bytes(int n, int P, bool accum)
{
    return phase_bytes<Store, K>(n) + (accum ? round16((size_t)n * K * 4) : 0) +
           round16((size_t)K * (P + 1) * 4) + round16((size_t)K * 20);
}

// ---------------------------------------------------------------- pair update
// Biased sign of eq. (4) on the minimum angular difference of d: +1 iff
// frac(d) < 1/2, i.e. iff floor(2d) is even. An FMA rounded toward -inf
// into the binade of 1.5 * 2^23 (ulp 1) gives 1.5 * 2^23 + floor(c d)
// exactly for |c d| < 2^22, and its last bit is the parity of floor(c d):
// one instruction for the whole decision, exact at the ties d = k / 2 too.
// c = -2 evaluates the sign of -d (the other orientation of the pair).
// Eq. (6) with J = -w is then, with s = sgn_b(x_i - x_j):
//   x_i <- x_i + alpha w s; x_j <- x_j - alpha w s (wrapped to [-1/2, 1/2]).
__device__ __forceinline__ uint32_t floor_parity(float c, float d)
{
    return __float_as_uint(__fmaf_rd(c, d, 12582912.0f)) & 1u;
}

// ---------------------------------------------------------------- DWT
// Dual window twist (Section II-D): windows [th - W/2, th + W/2) and their
// antipode; x is inside iff ((x - th + W/2) mod 1/2) < W. With y = 2x + c,
// c = 2 (W/2 - th) precomputed per replica, the test is frac(y) < 2W, i.e.
// floor(y) != floor(y - 2W): two adds rounded toward -inf into the binade
// of 1.5 * 2^23 give both floors, and they differ exactly for the phases
// inside (c2 = c - 2W is precomputed too).
__device__ __forceinline__ bool in_windows(float x, float c1, float c2)
{
    const float y1 = fmaf(2.0f, x, c1), y2 = fmaf(2.0f, x, c2);
    return __float_as_uint(__fadd_rd(y1, 12582912.0f)) != __float_as_uint(__fadd_rd(y2, 12582912.0f));
}

template <int K>
__device__ __forceinline__ void dwt_apply(float (&x)[K], const float *thc, const float *thc2, const float (&st)[K])
{
#pragma unroll
    for (int r = 0; r < K; ++r)
        if (in_windows(x[r], thc[r], thc2[r])) x[r] = wrap_c(__fadd_rn(x[r], st[r]));
}

// ---------------------------------------------------------------- segments
// Shared-memory layout of one tile and the per-segment prologue (bounded
// wait, init or load) and epilogue (readout, store, publish).
template <typename Store, int K>
struct Tile {
    Store *xs;     // [n][K] phases
    float *acc;    // [n][K] NO_SCS accumulators (mode 1 only)
    int *D;        // [K][P+1] readout difference arrays
    float *thc;    // [K] DWT offsets 2 (W/2 - theta)
    float *thc2;   // [K] the same minus 2W
    float *stp;    // [K] twist step of each replica (sign drawn or +1)
    int *imp;      // [K] readout: the replica's kept readout changed
    uint32_t *Bs;  // [K] readout: bisector position of the replica
    size_t vec_bytes;
};

template <typename Store, int K>
__device__ __forceinline__ Tile<Store, K> carve(unsigned char *smem, int n, int P, bool accum)
{
    Tile<Store, K> t;
    t.xs = reinterpret_cast<Store *>(smem);
    t.vec_bytes = phase_bytes<Store, K>(n);
    size_t off = t.vec_bytes;
    t.acc = reinterpret_cast<float *>(smem + off);
    if (accum) off += round16((size_t)n * K * 4);
    t.D = reinterpret_cast<int *>(smem + off);
    off += round16((size_t)K * (P + 1) * 4);
    t.thc = reinterpret_cast<float *>(smem + off);
    t.stp = t.thc + K;
    t.imp = reinterpret_cast<int *>(t.thc + 2 * K);
    t.Bs = reinterpret_cast<uint32_t *>(t.thc + 3 * K);
    t.thc2 = t.thc + 4 * K;
    return t;
}

// Returns false when the bounded wait gave up (the error word is set).
template <typename Store, int K>
__device__ bool seg_begin(const InstView &v, const Segment &sg, const Tile<Store, K> &t, int *s_skip,
                          int32_t *ready, int32_t *err, uint64_t wait_limit_ns)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        *s_skip = 0;
        if (sg.flags & SEG_WAIT) {
            const int need = (int)(sg.s_begin - 1);
            unsigned long long t0, t1;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            while (atomicAdd(&ready[sg.tile], 0) < need) {
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
                if (t1 - t0 > wait_limit_ns) {
                    atomicOr(err, 1);
                    *s_skip = 1;
                    break;
                }
                __nanosleep(2000);
            }
            __threadfence();
        }
    }
    __syncthreads();
    if (*s_skip) return false;
#ifdef COSM_CHECKS
    // the lattice passes address slots from Q and Wd alone: they must tile n
    // (four sublattices of Q slots, Q a whole number of rows); the tile must
    // be one of the run's
    if (tid == 0) {
        const bool bad_tile = sg.tile < 0 || (int64_t)sg.tile * K >= (int64_t)v.replicas + K - 1;
        const bool bad_lat = v.mode == MODE_LATTICE2D_ && (v.Q * 4 != v.n || v.Wd < 1 || v.Q % v.Wd != 0);
        if ((bad_tile || bad_lat) && v.check) atomicOr(v.check, 2);
    }
#endif
    const Store *gst = reinterpret_cast<const Store *>(v.state) + (size_t)sg.tile * v.state_tile_stride;
    if (sg.flags & SEG_INIT) {
        // Alg. 1 "Set x_i random": Philox keyed by seed, counter (v/4, r, 0, 0)
        const uint32_t rep0 = (uint32_t)sg.tile * K;
        const uint32_t k0 = (uint32_t)v.seed, k1 = (uint32_t)(v.seed >> 32);
        for (int k = tid; k < v.n * K; k += nt) {
            const int slot = k / K, r = k % K;
            const uint32_t ov = (uint32_t)v.orig_of[slot];
            uint32_t c[4] = {ov >> 2, rep0 + (uint32_t)r, 0u, 0u};
            philox4x32_10(c, k0, k1);
            const uint32_t lo = (ov & 1) ? c[1] : c[0], hi = (ov & 1) ? c[3] : c[2];
            const uint32_t word = (ov & 2) ? hi : lo;
            if constexpr (std::is_same<Store, uint16_t>::value) t.xs[k] = (uint16_t)(word >> 16);
            else if constexpr (sizeof(Store) == 4) t.xs[k] = u24_centered(word);
            else t.xs[k] = to_store<Store>(u24_centered(word));
        }
        // mid-anneal tracking keeps the lowest-energy readout of the trial
        if (v.track > 0 && v.energy && tid < K && rep0 + tid < (uint32_t)v.replicas)
            v.energy[rep0 + tid] = LLONG_MAX;
    } else if (sg.flags & SEG_LOAD) {
        const uint4 *src = reinterpret_cast<const uint4 *>(gst);
        uint4 *dst = reinterpret_cast<uint4 *>(t.xs);
        for (size_t k = tid; k < t.vec_bytes / 16; k += nt) dst[k] = __ldcg(src + k);
    }
    __syncthreads();
    return true;
}

// Bisector readout with exact integer cuts (Alg. 1 final loop). Spin of v
// at bisector p is [p < f_v] xor h_v, with h_v the top bit of
// q_v = floor(x_v 2^32) and f_v = #{p : floor(p 2^31 / P) <= q_v mod 2^31};
// an edge is therefore cut on one interval of p or on its complement, which
// a difference array over p accumulates exactly. With local fields the
// readout is the fixed half circle [-1/4, 1/4) turn around the reference
// phase 0 (s_v = +1 iff ((q_v + 2^30) mod 2^32) < 2^31), and the energy of
// eq. (1) adds the field term. Each replica's readout then replaces its
// kept one (keep_better: only if strictly lower in energy), its energy goes
// to trace[k] (k >= 0), and with tracking the spins of a replaced readout
// are saved as bits.
template <typename Store, int K>
__device__ __noinline__ void tile_readout(const InstView &a, int tile, const Tile<Store, K> &t, int k, bool keep_better)
{
    const int tid = threadIdx.x, nt = blockDim.x, P = a.P;
    const uint32_t rep0 = (uint32_t)tile * K;
    __syncthreads();
    for (int i = tid; i < K * (P + 1); i += nt) t.D[i] = 0;
    __syncthreads();
    const int m = __ldg(a.off + a.C);
    if (a.hv) {
        int cs[K], fs[K];
#pragma unroll
        for (int r = 0; r < K; ++r) cs[r] = fs[r] = 0;
        for (int e = tid; e < m; e += nt) {
            const uint32_t rec = load_rec(a, e);
            const int wv = (int)__ldg(a.w + e);
            uint32_t qis[K], qjs[K];
            ld_q32<Store, K>(t.xs + (size_t)(rec & 0xFFFFu) * K, qis);
            ld_q32<Store, K>(t.xs + (size_t)(rec >> 16) * K, qjs);
#pragma unroll
            for (int r = 0; r < K; ++r)
                if (((qis[r] + 0x40000000u) ^ (qjs[r] + 0x40000000u)) >> 31) cs[r] += wv;
        }
        for (int u = tid; u < a.n; u += nt) {
            const int hvu = __ldg(a.hv + u);
            uint32_t q[K];
            ld_q32<Store, K>(t.xs + (size_t)u * K, q);
#pragma unroll
            for (int r = 0; r < K; ++r) fs[r] += ((q[r] + 0x40000000u) >> 31) ? -hvu : hvu;
        }
#pragma unroll
        for (int r = 0; r < K; ++r) {
            int c = cs[r], f = fs[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
                f += __shfl_xor_sync(0xFFFFFFFFu, f, o);
            }
            if ((tid & 31) == 0) {
                if (c) atomicAdd(t.D + r * (P + 1), c);
                if (f) atomicAdd(t.D + r * (P + 1) + 1, f);
            }
        }
    } else {
        int base[K];
#pragma unroll
        for (int r = 0; r < K; ++r) base[r] = 0;
        for (int e = tid; e < m; e += nt) {
            const uint32_t rec = load_rec(a, e);
            const int wv = (int)__ldg(a.w + e);
            const int i = (int)(rec & 0xFFFFu), j = (int)(rec >> 16);
            uint32_t qis[K], qjs[K];
            ld_q32<Store, K>(t.xs + (size_t)i * K, qis);
            ld_q32<Store, K>(t.xs + (size_t)j * K, qjs);
#pragma unroll
            for (int r = 0; r < K; ++r) {
                const uint32_t qi = qis[r], qj = qjs[r];
                const int fi = (int)(((uint64_t)((qi & 0x7FFFFFFFu) + 1u) * (uint64_t)P + 0x7FFFFFFFull) >> 31);
                const int fj = (int)(((uint64_t)((qj & 0x7FFFFFFFu) + 1u) * (uint64_t)P + 0x7FFFFFFFull) >> 31);
                const int lo = min(fi, fj), hi = max(fi, fj);
                int *Dr = t.D + r * (P + 1);
                if ((qi >> 31) == (qj >> 31)) {
                    if (lo < hi) {  // cut for p in [lo, hi)
                        atomicAdd(Dr + lo, wv);
                        atomicAdd(Dr + hi, -wv);
                    }
                } else {  // cut for p in [0, lo) and [hi, P)
                    base[r] += wv;
                    if (lo < P) atomicAdd(Dr + lo, -wv);
                    if (hi < P) atomicAdd(Dr + hi, wv);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < K; ++r) {
            int b = base[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
            if ((tid & 31) == 0 && b) atomicAdd(t.D + r * (P + 1), b);
        }
    }
    __syncthreads();
    if (tid < K) {
        const uint32_t rep = rep0 + tid;
        const int *Dr = t.D + tid * (P + 1);
        long long cut, F = 0;
        int bp;
        uint32_t B;
        if (a.hv) {
            cut = Dr[0];
            F = Dr[1];
            bp = -1;
            B = 0xC0000000u;
        } else {
            long long accv = 0;
            cut = LLONG_MIN;
            bp = 0;
            for (int p = 0; p < P; ++p) {
                accv += Dr[p];
                if (accv > cut) { cut = accv; bp = p; }
            }
            B = (uint32_t)(((uint64_t)bp << 31) / (uint64_t)P);
        }
        int take = 0;
        if (rep < (uint32_t)a.replicas) {
            const long long E = a.W - 2 * cut - F;
            if (k >= 0 && a.trace) a.trace[(size_t)rep * a.n_trace + k] = E;
            // __ldcg: the value may come from a segment of this tile run on another SM
            take = !keep_better || !a.energy || E < __ldcg(a.energy + rep);
            if (take) {
                a.cut[rep] = cut;
                a.bestp[rep] = bp;
                if (a.energy) a.energy[rep] = E;
                if (a.bisB) a.bisB[rep] = B;
            }
        }
        t.imp[tid] = take;
        t.Bs[tid] = B;
    }
    if (!a.bits) return;
    __syncthreads();
    int any = 0;
#pragma unroll
    for (int r = 0; r < K; ++r) any |= t.imp[r];
    if (!any) return;
    uint32_t Bl[K];
#pragma unroll
    for (int r = 0; r < K; ++r) Bl[r] = t.Bs[r];
    for (int wi = tid; wi < a.words; wi += nt) {
        uint32_t word[K];
#pragma unroll
        for (int r = 0; r < K; ++r) word[r] = 0u;
        const int v0 = wi * 32, v1 = min(a.n, v0 + 32);
        for (int u = v0; u < v1; ++u) {
            uint32_t q[K];
            ld_q32<Store, K>(t.xs + (size_t)u * K, q);
#pragma unroll
            for (int r = 0; r < K; ++r)
                if ((uint32_t)(q[r] - Bl[r]) < 0x80000000u) word[r] |= 1u << (u - v0);
        }
#pragma unroll
        for (int r = 0; r < K; ++r)
            if (t.imp[r]) a.bits[(size_t)(rep0 + r) * a.words + wi] = word[r];
    }
    __syncthreads();  // the next sweep rewrites the phases read above
}

template <typename Store, int K>
__device__ void seg_end(const InstView &a, const Segment &sg, const Tile<Store, K> &t, int32_t *ready)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    // with tracking the readout after the last sweep ran inside the sweep loop
    if ((sg.flags & SEG_READOUT) && a.track <= 0) tile_readout<Store, K>(a, sg.tile, t, -1, false);
    if (sg.flags & SEG_STORE) {
        Store *gst = reinterpret_cast<Store *>(a.state) + (size_t)sg.tile * a.state_tile_stride;
        const uint4 *src = reinterpret_cast<const uint4 *>(t.xs);
        uint4 *dst = reinterpret_cast<uint4 *>(gst);
        for (size_t k = tid; k < t.vec_bytes / 16; k += nt) __stcg(dst + k, src[k]);
        __threadfence();
    }
    __syncthreads();
    if ((sg.flags & SEG_SIGNAL) && tid == 0) atomicExch(&ready[sg.tile], (int)sg.s_end);
}

// ---------------------------------------------------------------- sub-sweeps
// General graphs: colour c's edge records [off[c], off[c+1]) map to threads;
// each thread takes a batch of edges at a time (edges of one colour share no
// vertex, so all loads of a batch may precede its stores), which keeps
// several edge-record loads in flight (the batch sizes are given with each
// edge-list sweep below).
// An int8 weight as a float without the conversion unit: the bits of
// 1.5 * 2^23 + w, minus 1.5 * 2^23 (exact for |w| < 2^22).
__device__ __forceinline__ float weight_f(int8_t w)
{
    return __fadd_rn(__int_as_float(0x4B400000 + (int)w), -12582912.0f);
}

// Pair update inside a 2x2 block. x1, x2 are the block's slots; eq. (6)
// takes x_i as the endpoint with the smaller original id, which is x1
// except at a torus wrap. With d = x1 - x2 (any |d| < 2^21, so phases may
// stay unwrapped inside a sweep):
//     x_i = x1:  the step on x1 is +alpha w iff floor(2d) is even
//     x_i = x2:  the step on x1 is -alpha w iff floor(-2d) is even
// so a wrap edge passes c = -2 and aw = -alpha w, an ordinary one c = 2 and
// aw = alpha w, and both follow the oracle's biased sign exactly, ties
// included. Binary32 phases are wrapped to [-1/2, 1/2] at the end of the odd
// pass of every wrap_p-th sweep (every sweep for 16-bit storage): the host
// picks wrap_p so that the steps taken in between keep |g| < 1, where
// binary32 keeps an ulp of at most 2^-24 turn.
template <int K>
__device__ __forceinline__ void pair_fast(float (&x1)[K], float (&x2)[K], float aw, float c)
{
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const float d = __fadd_rn(x1[r], -x2[r]);
        const float st = floor_parity(c, d) ? -aw : aw;
        x1[r] = __fadd_rn(x1[r], st);
        x2[r] = __fadd_rn(x2[r], -st);
    }
}

// 16-bit float storage (binary16, bfloat16) in the lattice passes: a phase
// is stored once per pass of two colours, so it is wrapped and rounded to
// the storage type once, when its block is stored; the two updates in
// between are binary32.
template <typename Store, int K>
__device__ __forceinline__ void pair_block(float (&x1)[K], float (&x2)[K], float aw, float c)
{
    pair_fast<K>(x1, x2, aw, c);
}

template <int K>
__device__ __forceinline__ void wrap_all(float (&x)[K])
{
#pragma unroll
    for (int r = 0; r < K; ++r) x[r] = wrap_c(x[r]);
}

template <int K>
__device__ __forceinline__ void dwt_nowrap(float (&x)[K], const float *thc, const float *thc2, const float (&st)[K])
{
#pragma unroll
    for (int r = 0; r < K; ++r)
        if (in_windows(x[r], thc[r], thc2[r])) x[r] = __fadd_rn(x[r], st[r]);
}

// 2D torus in the sublattice layout: groups A = (even r, even c), B = (even,
// odd), C = (odd, even), D = (odd, odd), Q = n/4 slots each, row-major with
// Wd = L2/2 columns. With the colour order (even-column horizontal,
// even-row vertical, odd-column horizontal, odd-row vertical), colours 0
// and 1 act inside the 2x2 blocks {A[f], B[f], C[f], D[f]} and colours 2
// and 3 inside the shifted blocks {D[f], C[g(f)], B[h(f)], A[g(h(f))]},
// where g = next column (row wrap) and h = next row (torus wrap). A thread
// loads a block, applies both colours in registers and stores it: every
// vertex meets one edge of each colour inside its block. Edge indices are
// implicit; weights are +-1 bits.

__device__ __forceinline__ float signed_alpha(uint32_t wb, uint32_t bit, float alpha)
{
    return (wb & bit) ? -alpha : alpha;
}

// 1, 2 or 4 words at a 32-bit shared address.
template <int NW>
__device__ __forceinline__ void ld_words(uint32_t a, uint32_t (&w)[NW])
{
    if constexpr (NW == 1) {
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(w[0]) : "r"(a) : "memory");
    } else if constexpr (NW == 2) {
        asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "r"(a) : "memory");
    } else {
        static_assert(NW == 4, "NW");
        asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "r"(a) : "memory");
    }
}
template <int NW>
__device__ __forceinline__ void st_words(uint32_t a, const uint32_t (&w)[NW])
{
    if constexpr (NW == 1) {
        asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(w[0]) : "memory");
    } else if constexpr (NW == 2) {
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(w[0]), "r"(w[1]) : "memory");
    } else {
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                     "r"(w[3]) : "memory");
    }
}
// A slot's K phases in the storage type at a 32-bit shared address, as
// binary32 (ldk / stk by address).
template <typename Store, int K>
__device__ __forceinline__ void lds_k(uint32_t a, float (&x)[K])
{
    constexpr int NW = (int)(sizeof(Store) * K / 4);
    uint32_t w[NW];
    ld_words<NW>(a, w);
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        if constexpr (sizeof(Store) == 4) {
            x[i] = __uint_as_float(w[i]);
        } else {
            const float2 f = h2_to_f2<Store>(w[i]);
            x[2 * i] = f.x;
            x[2 * i + 1] = f.y;
        }
    }
}
template <typename Store, int K>
__device__ __forceinline__ void sts_k(uint32_t a, const float (&x)[K])
{
    constexpr int NW = (int)(sizeof(Store) * K / 4);
    uint32_t w[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        if constexpr (sizeof(Store) == 4) w[i] = __float_as_uint(x[i]);
        else w[i] = f2_to_h2<Store>(x[2 * i], x[2 * i + 1]);
    }
    st_words<NW>(a, w);
}

template <typename Store, int K>
__device__ __forceinline__ void block_pass_even(Store *xs, const uint8_t *wnib, float alpha, int Q)
{
    constexpr uint32_t E = sizeof(Store) * K;  // bytes per slot
    const uint32_t qb = (uint32_t)Q * E, qb2 = 2 * qb, qb3 = 3 * qb, step = blockDim.x * E;
    uint32_t ad = (uint32_t)__cvta_generic_to_shared(xs) + threadIdx.x * E;
#pragma unroll 2
    for (int f = threadIdx.x; f < Q; f += blockDim.x, ad += step) {
        const uint32_t wb = __ldg(wnib + f);
        float xa[K], xb[K], xc[K], xd[K];
        lds_k<Store, K>(ad, xa);
        lds_k<Store, K>(ad + qb, xb);
        lds_k<Store, K>(ad + qb2, xc);
        lds_k<Store, K>(ad + qb3, xd);
        // colour 0: A-B, C-D; colour 1: A-C, B-D (first slot = smaller id)
        pair_block<Store, K>(xa, xb, signed_alpha(wb, 1u, alpha), 2.0f);
        pair_block<Store, K>(xc, xd, signed_alpha(wb, 2u, alpha), 2.0f);
        pair_block<Store, K>(xa, xc, signed_alpha(wb, 4u, alpha), 2.0f);
        pair_block<Store, K>(xb, xd, signed_alpha(wb, 8u, alpha), 2.0f);
        // binary32 phases stay unwrapped until the next wrapping odd pass;
        // 16-bit phases are wrapped and rounded by their store
        if constexpr (sizeof(Store) == 2) {
            wrap_all<K>(xa); wrap_all<K>(xb); wrap_all<K>(xc); wrap_all<K>(xd);
        }
        sts_k<Store, K>(ad, xa);
        sts_k<Store, K>(ad + qb, xb);
        sts_k<Store, K>(ad + qb2, xc);
        sts_k<Store, K>(ad + qb3, xd);
    }
}

// kFixedColumn: the thread count is a multiple of Wd, so every block a
// thread visits sits in the same column and the column wrap is fixed.
template <typename Store, int K, bool kFixedColumn, bool kWrap>
__device__ __forceinline__ void block_pass_odd(Store *xs, const uint8_t *wnib, float alpha, int Q, int Wd,
                                               int m0, int dm, bool dwt, const float *thc, const float *thc2,
                                               const float *stp)
{
    float st[K];  // the twist step of each replica
#pragma unroll
    for (int r = 0; r < K; ++r) st[r] = dwt ? stp[r] : 0.0f;
    // byte offsets from D[f] to C[g], B[h], A[gh] (g: next column, h: next row)
    constexpr uint32_t E = sizeof(Store) * K;  // bytes per slot
    const uint32_t qb = (uint32_t)Q * E, wdb = (uint32_t)Wd * E, rowwrap = (uint32_t)(Wd - Q) * E;
    const uint32_t step = blockDim.x * E;
    uint32_t ad = (uint32_t)__cvta_generic_to_shared(xs) + 3 * qb + threadIdx.x * E;
    int m = m0;  // column of block f within its row
    const bool cw0 = (m0 == Wd - 1);
    const uint32_t goffb0 = cw0 ? (uint32_t)(1 - Wd) * E : E;
#pragma unroll 2
    for (int f = threadIdx.x; f < Q; f += blockDim.x, ad += step) {
        uint32_t goffb = goffb0;
        bool cw = cw0;
        if (!kFixedColumn) {
            cw = (m == Wd - 1);  // next column wraps to column 0
            goffb = cw ? (uint32_t)(1 - Wd) * E : E;
            m += dm;
            if (m >= Wd) m -= Wd;
        }
        const bool rw = (f >= Q - Wd);      // next row wraps to row 0
        const uint32_t hoffb = rw ? rowwrap : wdb;
        const uint32_t aC = ad - qb + goffb, aB = ad - 2 * qb + hoffb, aA = ad - 3 * qb + goffb + hoffb;
        // wrap edges: the other orientation (c = -2, negated step)
        const float tzc = cw ? -2.0f : 2.0f, tzr = rw ? -2.0f : 2.0f;
        const uint32_t wb = __ldg(wnib + Q + f) ^ (cw ? 3u : 0u) ^ (rw ? 12u : 0u);
        float xd[K], xc[K], xb[K], xa[K];
        lds_k<Store, K>(ad, xd);
        lds_k<Store, K>(aC, xc);
        lds_k<Store, K>(aB, xb);
        lds_k<Store, K>(aA, xa);
        // colour 2: D-C, B-A (horizontal from odd columns)
        pair_block<Store, K>(xd, xc, signed_alpha(wb, 1u, alpha), tzc);
        pair_block<Store, K>(xb, xa, signed_alpha(wb, 2u, alpha), tzc);
        // colour 3: D-B, C-A (vertical from odd rows)
        pair_block<Store, K>(xd, xb, signed_alpha(wb, 4u, alpha), tzr);
        pair_block<Store, K>(xc, xa, signed_alpha(wb, 8u, alpha), tzr);
        if (dwt) {
            // the DWT follows the last colour of the sweep; every vertex is in
            // exactly one shifted block
            if constexpr (sizeof(Store) == 4) {
                dwt_nowrap<K>(xd, thc, thc2, st);
                dwt_nowrap<K>(xc, thc, thc2, st);
                dwt_nowrap<K>(xb, thc, thc2, st);
                dwt_nowrap<K>(xa, thc, thc2, st);
            } else {
                dwt_apply<K>(xd, thc, thc2, st);
                dwt_apply<K>(xc, thc, thc2, st);
                dwt_apply<K>(xb, thc, thc2, st);
                dwt_apply<K>(xa, thc, thc2, st);
            }
        }
        if constexpr (kWrap || sizeof(Store) == 2) {
            wrap_all<K>(xa); wrap_all<K>(xb); wrap_all<K>(xc); wrap_all<K>(xd);
        }
        sts_k<Store, K>(ad, xd);
        sts_k<Store, K>(aC, xc);
        sts_k<Store, K>(aB, xb);
        sts_k<Store, K>(aA, xa);
    }
}

// ---------------------------------------------------------------- paired binary32
// Two replicas' binary32 phases in one 64-bit register pair, updated with the
// packed f32x2 instructions of sm_100 and later: one issue slot carries two
// binary32 additions, each rounded exactly as the scalar instruction, so the
// paired passes give bit-identical phases to the scalar ones above.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 p_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 p_sub(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 p_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float p_lo(f32x2 v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float p_hi(f32x2 v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ f32x2 p_fma_rd(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
constexpr f32x2 kMagic2 = 0x4B4000004B400000ull;  // 1.5 * 2^23 in both lanes
constexpr f32x2 kTwo2 = 0x4000000040000000ull;    // 2 in both lanes
constexpr f32x2 kMinusTwo2 = 0xC0000000C0000000ull;
__device__ __forceinline__ f32x2 p_wrap(f32x2 v) { return p_sub(v, p_sub(p_add(v, kMagic2), kMagic2)); }

// aw with its sign flipped where t is odd: aw + t 2^31 mod 2^32 (an integer
// multiply-add, issued to the FMA pipe rather than the logic unit).
__device__ __forceinline__ uint32_t flip_if_odd(uint32_t aw, uint32_t t)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, 0x80000000, %2;" : "=r"(r) : "r"(t), "r"(aw));
    return r;
}

// The same sign flip on the logic pipe: aw xor (t << 31) (a funnel shift
// and an xor), for kernels whose FMA pipe is the busier one.
__device__ __forceinline__ uint32_t flip_if_odd_alu(uint32_t aw, uint32_t t)
{
    uint32_t s;
    asm("shf.l.clamp.b32 %0, 0, %1, 31;" : "=r"(s) : "r"(t));
    return aw ^ s;
}

// Pair update of eq. (6) as pair_fast, for two replicas: t = 1.5 * 2^23 +
// floor(c d) per lane (one fma rounded toward -inf), and the step on x1 is
// aw (the bits of alpha w, shared by both lanes), negated where floor(c d)
// is odd. kAluLanes of the two lanes take the flip on the logic pipe (the
// 16-bit lattice passes, FMA-bound by their conversions: binary16 +4.6 %,
// bfloat16 +1.4 % with one lane; binary32 loses 2-6 %, so it keeps both on
// the FMA pipe).
template <int kAluLanes = 0>
__device__ __forceinline__ void pair_x2(f32x2 &x1, f32x2 &x2, f32x2 aw2, f32x2 c2)
{
    const f32x2 d = p_sub(x1, x2);
    const f32x2 t = p_fma_rd(c2, d, kMagic2);
    const uint32_t hi = kAluLanes >= 1 ? flip_if_odd_alu((uint32_t)(aw2 >> 32), (uint32_t)(t >> 32))
                                       : flip_if_odd((uint32_t)(aw2 >> 32), (uint32_t)(t >> 32));
    const uint32_t lo = kAluLanes >= 2 ? flip_if_odd_alu((uint32_t)aw2, (uint32_t)t)
                                       : flip_if_odd((uint32_t)aw2, (uint32_t)t);
    const f32x2 st = ((f32x2)hi << 32) | lo;
    x1 = p_add(x1, st);
    x2 = p_sub(x2, st);
}

template <int K>
__device__ __forceinline__ void ldp(const float *p, f32x2 (&x)[K / 2])
{
    if constexpr (K == 2) {
        x[0] = *reinterpret_cast<const f32x2 *>(p);
    } else {
        static_assert(K == 4, "K");
        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
        x[0] = v.x;
        x[1] = v.y;
    }
}
template <int K>
__device__ __forceinline__ void stp(float *p, const f32x2 (&x)[K / 2])
{
    if constexpr (K == 2) {
        *reinterpret_cast<f32x2 *>(p) = x[0];
    } else {
        *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(x[0], x[1]);
    }
}

// The dual window twist of dwt_nowrap for two replicas: the floors of
// y1 = 2x + c and y2 = 2x + c - 2W per lane (fma, then an add rounded toward
// -inf into the binade of 1.5 * 2^23); their difference, exact in binary32
// (1 inside, 0 outside), scales the lane's step in one fma: x + st rounded
// once inside, x + 0 outside.
__device__ __forceinline__ f32x2 p_add_rd(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ void dwt_x2(f32x2 &x, f32x2 c1, f32x2 c2, f32x2 st2)
{
    const f32x2 k1 = p_add_rd(p_fma(kTwo2, x, c1), kMagic2);
    const f32x2 k2 = p_add_rd(p_fma(kTwo2, x, c2), kMagic2);
    x = p_fma(p_sub(k1, k2), st2, x);
}

// Shared-memory loads and stores of a slot's K/2 replica pairs at a 32-bit
// shared address (per-thread addresses advance by adds; no 64-bit index math).
template <int K>
__device__ __forceinline__ void lds_p(uint32_t a, f32x2 (&x)[K / 2])
{
    if constexpr (K == 2) {
        asm volatile("ld.shared.b64 %0, [%1];" : "=l"(x[0]) : "r"(a) : "memory");
    } else {
        static_assert(K == 4, "K");
        asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(x[0]), "=l"(x[1]) : "r"(a) : "memory");
    }
}
template <int K>
__device__ __forceinline__ void sts_p(uint32_t a, const f32x2 (&x)[K / 2])
{
    if constexpr (K == 2) {
        asm volatile("st.shared.b64 [%0], %1;" ::"r"(a), "l"(x[0]) : "memory");
    } else {
        asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(a), "l"(x[0]), "l"(x[1]) : "memory");
    }
}

template <int K>
__device__ __forceinline__ void block_pass_even_x2(float *xs, const uint8_t *wnib, float alpha, int Q)
{
    constexpr uint32_t E = K * 4;  // bytes per slot
    const uint32_t a1 = __float_as_uint(alpha), n1 = a1 ^ 0x80000000u;
    const uint32_t qb = (uint32_t)Q * E, qb2 = 2 * qb, qb3 = 3 * qb, step = blockDim.x * E;
    uint32_t ad = (uint32_t)__cvta_generic_to_shared(xs) + threadIdx.x * E;
#pragma unroll 2
    for (int f = threadIdx.x; f < Q; f += blockDim.x, ad += step) {
        const uint32_t wb = __ldg(wnib + f);
        f32x2 xa[K / 2], xb[K / 2], xc[K / 2], xd[K / 2];
        lds_p<K>(ad, xa);
        lds_p<K>(ad + qb, xb);
        lds_p<K>(ad + qb2, xc);
        lds_p<K>(ad + qb3, xd);
        const f32x2 a2 = ((f32x2)a1 << 32) | a1, n2 = ((f32x2)n1 << 32) | n1;
        const f32x2 w0 = (wb & 1u) ? n2 : a2, w1 = (wb & 2u) ? n2 : a2;
        const f32x2 w2 = (wb & 4u) ? n2 : a2, w3 = (wb & 8u) ? n2 : a2;
#pragma unroll
        for (int h = 0; h < K / 2; ++h) {
            pair_x2(xa[h], xb[h], w0, kTwo2);
            pair_x2(xc[h], xd[h], w1, kTwo2);
            pair_x2(xa[h], xc[h], w2, kTwo2);
            pair_x2(xb[h], xd[h], w3, kTwo2);
        }
        sts_p<K>(ad, xa);
        sts_p<K>(ad + qb, xb);
        sts_p<K>(ad + qb2, xc);
        sts_p<K>(ad + qb3, xd);
    }
}

// One shifted block {D[f], C[g], B[h], A[gh]} of the odd pass for two or four
// replicas; kRowWrap: f sits in the last block row, so h wraps to row 0;
// kDwt: the twist follows the colours; kWrap: the phases are wrapped to
// [-1/2, 1/2] before the store.
template <int K, bool kRowWrap, bool kDwt, bool kWrap>
__device__ __forceinline__ void odd_block_x2(uint32_t ad, uint32_t oC, uint32_t oB, uint32_t oA, uint32_t wb,
                                             uint32_t a1, f32x2 tzc, const f32x2 (&th2)[K / 2],
                                             const f32x2 (&tk2)[K / 2], const f32x2 (&st2)[K / 2])
{
    // wrap edges: the other orientation (c = -2, negated step)
    constexpr f32x2 tzr = kRowWrap ? kMinusTwo2 : kTwo2;
    const uint32_t n1 = a1 ^ 0x80000000u;
    f32x2 xd[K / 2], xc[K / 2], xb[K / 2], xa[K / 2];
    lds_p<K>(ad, xd);
    lds_p<K>(ad + oC, xc);
    lds_p<K>(ad + oB, xb);
    lds_p<K>(ad + oA, xa);
    const f32x2 a2 = ((f32x2)a1 << 32) | a1, n2 = ((f32x2)n1 << 32) | n1;
    const f32x2 w0 = (wb & 1u) ? n2 : a2, w1 = (wb & 2u) ? n2 : a2;
    const f32x2 w2 = (wb & 4u) ? n2 : a2, w3 = (wb & 8u) ? n2 : a2;
#pragma unroll
    for (int h = 0; h < K / 2; ++h) {
        // colour 2: D-C, B-A; colour 3: D-B, C-A
        pair_x2(xd[h], xc[h], w0, tzc);
        pair_x2(xb[h], xa[h], w1, tzc);
        pair_x2(xd[h], xb[h], w2, tzr);
        pair_x2(xc[h], xa[h], w3, tzr);
        if constexpr (kDwt) {
            dwt_x2(xd[h], th2[h], tk2[h], st2[h]);
            dwt_x2(xc[h], th2[h], tk2[h], st2[h]);
            dwt_x2(xb[h], th2[h], tk2[h], st2[h]);
            dwt_x2(xa[h], th2[h], tk2[h], st2[h]);
        }
        if constexpr (kWrap) {
            xa[h] = p_wrap(xa[h]);
            xb[h] = p_wrap(xb[h]);
            xc[h] = p_wrap(xc[h]);
            xd[h] = p_wrap(xd[h]);
        }
    }
    sts_p<K>(ad, xd);
    sts_p<K>(ad + oC, xc);
    sts_p<K>(ad + oB, xb);
    sts_p<K>(ad + oA, xa);
}

// The odd pass: blocks above the last block row first (fixed offsets to the
// next row), then the last row, whose next row wraps to row 0.
template <int K, bool kFixedColumn, bool kDwt, bool kWrap>
__device__ __forceinline__ void block_pass_odd_x2(float *xs, const uint8_t *wnib, float alpha, int Q, int Wd,
                                                  int m0, int dm, const float *thc, const float *thc2,
                                                  const float *stp_)
{
    constexpr uint32_t E = K * 4;  // bytes per slot
    const uint32_t a1 = __float_as_uint(alpha);
    f32x2 th2[K / 2], tk2[K / 2], st2[K / 2];
#pragma unroll
    for (int h = 0; h < K / 2; ++h) {
        th2[h] = kDwt ? (((f32x2)__float_as_uint(thc[2 * h + 1]) << 32) | __float_as_uint(thc[2 * h])) : 0ull;
        tk2[h] = kDwt ? (((f32x2)__float_as_uint(thc2[2 * h + 1]) << 32) | __float_as_uint(thc2[2 * h])) : 0ull;
        st2[h] = kDwt ? (((f32x2)__float_as_uint(stp_[2 * h + 1]) << 32) | __float_as_uint(stp_[2 * h])) : 0ull;
    }
    // byte offsets from D[f] (sublattice D at 3Q) to C[g], B[h], A[gh] with
    // g = f + goff (next column) and h = f + hoff (next row)
    const uint32_t qb = (uint32_t)Q * E;
    const uint32_t wdb = (uint32_t)Wd * E;
    const uint32_t rowwrap = (uint32_t)(Wd - Q) * E;  // hoff at the last row, mod 2^32
    const uint32_t step = blockDim.x * E;
    uint32_t ad = (uint32_t)__cvta_generic_to_shared(xs) + 3 * qb + threadIdx.x * E;
    int m = m0;  // column of block f within its row
    bool cw = (m0 == Wd - 1);  // next column wraps to column 0
    uint32_t goffb = cw ? (uint32_t)(1 - Wd) * E : E;
    const int qlast = Q - Wd;  // first block of the last row
    int f = threadIdx.x;
#pragma unroll 5
    for (; f < qlast; f += blockDim.x, ad += step) {
        if (!kFixedColumn) {
            cw = (m == Wd - 1);
            goffb = cw ? (uint32_t)(1 - Wd) * E : E;
            m += dm;
            if (m >= Wd) m -= Wd;
        }
        const uint32_t wb = __ldg(wnib + Q + f) ^ (cw ? 3u : 0u);
        odd_block_x2<K, false, kDwt, kWrap>(ad, goffb - qb, wdb - 2 * qb, goffb + wdb - 3 * qb, wb, a1,
                                            cw ? kMinusTwo2 : kTwo2, th2, tk2, st2);
    }
    for (; f < Q; f += blockDim.x, ad += step) {
        if (!kFixedColumn) {
            cw = (m == Wd - 1);
            goffb = cw ? (uint32_t)(1 - Wd) * E : E;
            m += dm;
            if (m >= Wd) m -= Wd;
        }
        const uint32_t wb = __ldg(wnib + Q + f) ^ (cw ? 3u : 0u) ^ 12u;
        odd_block_x2<K, true, kDwt, kWrap>(ad, goffb - qb, rowwrap - 2 * qb, goffb + rowwrap - 3 * qb, wb, a1,
                                           cw ? kMinusTwo2 : kTwo2, th2, tk2, st2);
    }
}

template <int K, bool kFixedColumn>
__device__ __forceinline__ void block_pass_odd_x2_sel(float *xs, const uint8_t *wnib, float alpha, int Q, int Wd,
                                                      int m0, int dm, bool dwt, bool wrap, const float *thc,
                                                      const float *thc2, const float *stp_)
{
    if (dwt) {
        if (wrap) block_pass_odd_x2<K, kFixedColumn, true, true>(xs, wnib, alpha, Q, Wd, m0, dm, thc, thc2, stp_);
        else block_pass_odd_x2<K, kFixedColumn, true, false>(xs, wnib, alpha, Q, Wd, m0, dm, thc, thc2, stp_);
    } else {
        if (wrap) block_pass_odd_x2<K, kFixedColumn, false, true>(xs, wnib, alpha, Q, Wd, m0, dm, thc, thc2, stp_);
        else block_pass_odd_x2<K, kFixedColumn, false, false>(xs, wnib, alpha, Q, Wd, m0, dm, thc, thc2, stp_);
    }
}

// Block pairs in the even pass (two replicas per tile, an even number of
// block columns): a thread takes the blocks f = 2u and f + 1 of one block row
// together, so the slots of both sit side by side in each sublattice and move
// in 16-byte shared accesses, with one weight load, one address update and
// one loop step per two blocks. (In the odd pass the C and A slots of such a
// pair straddle a 16-byte boundary; their 8-byte accesses at a 16-byte
// stride conflict in the shared-memory banks, so the odd pass keeps one
// block per thread.)
__device__ __forceinline__ void lds_q2(uint32_t a, f32x2 &x0, f32x2 &x1)
{
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(x0), "=l"(x1) : "r"(a) : "memory");
}
__device__ __forceinline__ void sts_q2(uint32_t a, f32x2 x0, f32x2 x1)
{
    asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(a), "l"(x0), "l"(x1) : "memory");
}

__device__ __forceinline__ void block_pass_even_x2p(float *xs, const uint8_t *wnib, float alpha, int Q)
{
    constexpr uint32_t E = 8;  // bytes per slot (two binary32 replicas)
    const uint32_t a1 = __float_as_uint(alpha), n1 = a1 ^ 0x80000000u;
    const f32x2 a2 = ((f32x2)a1 << 32) | a1, n2 = ((f32x2)n1 << 32) | n1;
    const uint32_t qb = (uint32_t)Q * E, qb2 = 2 * qb, qb3 = 3 * qb, step = blockDim.x * 2 * E;
    const int U = Q >> 1;
    const unsigned short *wp = reinterpret_cast<const unsigned short *>(wnib);
    uint32_t ad = (uint32_t)__cvta_generic_to_shared(xs) + threadIdx.x * 2 * E;
#pragma unroll 1
    for (int u = threadIdx.x; u < U; u += blockDim.x, ad += step) {
        const uint32_t wb = __ldg(wp + u);  // block 2u: bits 0-3, block 2u + 1: bits 8-11
        f32x2 xa0, xa1, xb0, xb1, xc0, xc1, xd0, xd1;
        lds_q2(ad, xa0, xa1);
        lds_q2(ad + qb, xb0, xb1);
        lds_q2(ad + qb2, xc0, xc1);
        lds_q2(ad + qb3, xd0, xd1);
        // colour 0: A-B, C-D; colour 1: A-C, B-D (first slot = smaller id)
        pair_x2(xa0, xb0, (wb & 0x001u) ? n2 : a2, kTwo2);
        pair_x2(xa1, xb1, (wb & 0x100u) ? n2 : a2, kTwo2);
        pair_x2(xc0, xd0, (wb & 0x002u) ? n2 : a2, kTwo2);
        pair_x2(xc1, xd1, (wb & 0x200u) ? n2 : a2, kTwo2);
        pair_x2(xa0, xc0, (wb & 0x004u) ? n2 : a2, kTwo2);
        pair_x2(xa1, xc1, (wb & 0x400u) ? n2 : a2, kTwo2);
        pair_x2(xb0, xd0, (wb & 0x008u) ? n2 : a2, kTwo2);
        pair_x2(xb1, xd1, (wb & 0x800u) ? n2 : a2, kTwo2);
        sts_q2(ad, xa0, xa1);
        sts_q2(ad + qb, xb0, xb1);
        sts_q2(ad + qb2, xc0, xc1);
        sts_q2(ad + qb3, xd0, xd1);
    }
}

// ---------------------------------------------------------------- paired edge lists
// The edge-list sweep of binary32 tiles in f32x2 lanes: the two lanes of an
// instruction carry the two replicas of a pair (tiles of 2 or 4 replicas) or
// two edges of a thread's batch (single-replica tiles); each lane rounds
// every operation as the scalar instruction does and the wrap cadence below
// is the same for every tile size, so every tile size gives the same phases.
// Slots are addressed by 32-bit shared offsets; a batch past the end of its
// colour loads slot 0 harmlessly and skips its stores.
// kWrapEach: every update is wrapped (instances whose steps per sweep could
// carry a phase far from [-1/2, 1/2]); otherwise the phases are wrapped by the
// pass after the colours on every wrap_p-th sweep.
__device__ __forceinline__ float lds_f(uint32_t a)
{
    float x;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x) : "r"(a) : "memory");
    return x;
}
__device__ __forceinline__ void sts_f(uint32_t a, float x)
{
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(x) : "memory");
}
__device__ __forceinline__ f32x2 p_pack(float lo, float hi)
{
    return ((f32x2)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}

// One batch of B edges per thread (edges e0, e0 + nt, ...); kTail: the batch
// may run past the end e1 of its colour (loads of slot 0, stores skipped).
// kStaged: the colour's records sit in shared memory (edge e's record at
// sij + 4 e, its weight at sw + e), else they are read from global memory.
// kSgn: the records of a.ijs, whose bit 0 is the sign of a +-1 weight, so
// alpha w is alpha + bit 0 * 2^31 in integer arithmetic (the sign bit
// flipped; no weight load or conversion).
template <int K, int B, bool kWrapEach, bool kTail, bool kStaged = false, bool kSgn = false>
__device__ __forceinline__ void edge_batch_x2(const InstView &a, uint32_t xb, float alpha, int e0, int e1, int nt,
                                              uint32_t sij = 0, uint32_t sw = 0)
{
    static_assert(!(kStaged && kSgn), "staged records carry their weights apart");
    constexpr uint32_t E = K * 4;  // bytes per slot
    uint32_t ai[B], aj[B];
    float aw[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int e = e0 + u * nt;
        uint32_t rec = 0;
        int w = 0;
        if (!kTail || e < e1) {
            if constexpr (kStaged) {
                asm volatile("ld.shared.b32 %0, [%1];" : "=r"(rec) : "r"(sij + 4u * (uint32_t)e) : "memory");
                asm volatile("ld.shared.s8 %0, [%1];" : "=r"(w) : "r"(sw + (uint32_t)e) : "memory");
                rec = checked_rec(a, rec);
            } else if constexpr (kSgn) {
                rec = load_rec_sgn(a, e);
            } else {
                rec = load_rec(a, e);
                w = __ldg(a.w + e);
            }
        }
        aj[u] = xb + (rec >> 16) * E;
        if constexpr (kSgn) {
            ai[u] = xb + (rec & 0xFFFEu) * (E / 2);
            aw[u] = __uint_as_float(flip_if_odd(__float_as_uint(alpha), rec));
        } else {
            ai[u] = xb + (rec & 0xFFFFu) * E;
            aw[u] = alpha * weight_f((int8_t)w);
        }
    }
    if constexpr (K == 1) {
        float xi[B], xj[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            xi[u] = lds_f(ai[u]);
            xj[u] = lds_f(aj[u]);
        }
#pragma unroll
        for (int q = 0; q < B; q += 2) {
            f32x2 x1 = p_pack(xi[q], xi[q + 1]), x2 = p_pack(xj[q], xj[q + 1]);
            pair_x2(x1, x2, p_pack(aw[q], aw[q + 1]), kTwo2);
            if constexpr (kWrapEach) {
                x1 = p_wrap(x1);
                x2 = p_wrap(x2);
            }
            xi[q] = p_lo(x1);
            xi[q + 1] = p_hi(x1);
            xj[q] = p_lo(x2);
            xj[q + 1] = p_hi(x2);
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (!kTail || e0 + u * nt < e1) {
                sts_f(ai[u], xi[u]);
                sts_f(aj[u], xj[u]);
            }
        }
    } else {
        f32x2 xi[B][K / 2], xj[B][K / 2];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            lds_p<K>(ai[u], xi[u]);
            lds_p<K>(aj[u], xj[u]);
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const f32x2 aw2 = p_pack(aw[u], aw[u]);
#pragma unroll
            for (int h = 0; h < K / 2; ++h) {
                pair_x2(xi[u][h], xj[u][h], aw2, kTwo2);
                if constexpr (kWrapEach) {
                    xi[u][h] = p_wrap(xi[u][h]);
                    xj[u][h] = p_wrap(xj[u][h]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (!kTail || e0 + u * nt < e1) {
                sts_p<K>(ai[u], xi[u]);
                sts_p<K>(aj[u], xj[u]);
            }
        }
    }
}

// The colours of one sweep: whole batches without bounds checks, then at
// most one checked batch per thread at the end of each colour. (Trimming
// that last batch to the ceil(rem / nt) slots the block's remaining rem
// edges need cost 3-6 % on G(n, m) graphs: more code for little saving.)
template <int K, int B, bool kWrapEach, bool kSgn = false>
__device__ __forceinline__ void general_colours_x2(const InstView &a, float *xs, float alpha)
{
    static_assert(K == 1 || K == 2 || K == 4, "K");
    static_assert(K > 1 || B % 2 == 0, "B");
    const int nt = blockDim.x;
    const uint32_t xb = (uint32_t)__cvta_generic_to_shared(xs);
    for (int c = 0; c < a.C; ++c) {
        const int e1 = __ldg(a.off + c + 1);
        int e0 = __ldg(a.off + c) + threadIdx.x;
        for (; e0 + (B - 1) * nt < e1; e0 += B * nt)
            edge_batch_x2<K, B, kWrapEach, false, false, kSgn>(a, xb, alpha, e0, e1, nt);
        if (e0 < e1) edge_batch_x2<K, B, kWrapEach, true, false, kSgn>(a, xb, alpha, e0, e1, nt);
        __syncthreads();
    }
}

// Edge records staged in shared memory: while colour c runs, colour c + 1's
// records (packed slots and weights) stream into the other of two buffers
// with cp.async (16-byte chunks, cached in L2 only), so a colour's record
// loads are shared-memory loads instead of global loads on the critical
// path. A buffer holds the 16-byte chunks that cover the colour: records
// from off[c] rounded down to a multiple of 4, weights from off[c] rounded
// down to a multiple of 16 (the device arrays are padded so the chunks after
// the last colour exist).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void stage_colour(const InstView &a, int c, uint32_t buf)
{
    const int e0 = __ldg(a.off + c), e1 = __ldg(a.off + c + 1);
    const int i0 = e0 & ~3, i1 = (e1 + 3) & ~3;
    const int w0 = e0 & ~15, w1 = (e1 + 15) & ~15;
    const int nij = (i1 - i0) >> 2, nw = (w1 - w0) >> 4;
    const uint32_t bw = buf + (uint32_t)a.stage_ij;
    for (int k = threadIdx.x; k < nij + nw; k += blockDim.x) {
        if (k < nij) cp_async16(buf + 16u * (uint32_t)k, a.ij + i0 + 4 * k);
        else cp_async16(bw + 16u * (uint32_t)(k - nij), a.w + w0 + 16 * (k - nij));
    }
    cp_async_commit();
}

// The colours of one sweep with staged records. `cur` is the buffer that
// holds colour 0's records (staged by the previous sweep, or here when
// `first`); the last colour stages colour 0 of the next sweep unless `last`.
template <int K, int B, bool kWrapEach>
__device__ __forceinline__ void general_colours_x2s(const InstView &a, float *xs, float alpha, uint32_t stage,
                                                    bool first, bool last, int &cur)
{
    static_assert(K == 1 || K == 2 || K == 4, "K");
    static_assert(K > 1 || B % 2 == 0, "B");
    const int nt = blockDim.x;
    const uint32_t xb = (uint32_t)__cvta_generic_to_shared(xs);
    const uint32_t SB = (uint32_t)(a.stage_ij + a.stage_w);
    if (first) {
        stage_colour(a, 0, stage + (uint32_t)cur * SB);
        cp_async_wait_all();
        __syncthreads();
    }
    for (int c = 0; c < a.C; ++c) {
        if (c + 1 < a.C) stage_colour(a, c + 1, stage + (uint32_t)(cur ^ 1) * SB);
        else if (!last) stage_colour(a, 0, stage + (uint32_t)(cur ^ 1) * SB);
        const int ec = __ldg(a.off + c), e1 = __ldg(a.off + c + 1);
        const uint32_t buf = stage + (uint32_t)cur * SB;
        const uint32_t sij = buf - 4u * (uint32_t)(ec & ~3);
        const uint32_t sw = buf + (uint32_t)a.stage_ij - (uint32_t)(ec & ~15);
        int e0 = ec + threadIdx.x;
        for (; e0 + (B - 1) * nt < e1; e0 += B * nt)
            edge_batch_x2<K, B, kWrapEach, false, true>(a, xb, alpha, e0, e1, nt, sij, sw);
        if (e0 < e1) edge_batch_x2<K, B, kWrapEach, true, true>(a, xb, alpha, e0, e1, nt, sij, sw);
        cp_async_wait_all();
        __syncthreads();
        cur ^= 1;
    }
}

// The twist and / or the wrap of binary32 edge-list tiles after the colours,
// in f32x2 words: a word holds replicas 2h, 2h + 1 of one slot (K >= 2) or
// one replica of two slots (K = 1). The twist is dwt_x2 (the step is added
// without a wrap); kWrap wraps every phase.
template <int K, bool kDwt, bool kWrap>
__device__ __forceinline__ void twist_wrap_x2(float *xs, int n, const float *thc, const float *thc2,
                                              const float *stp_)
{
    constexpr int H = K >= 2 ? K / 2 : 1;  // words per slot (K = 1: a word spans two slots)
    f32x2 th2[H], tk2[H], st2[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int r0 = K >= 2 ? 2 * h : 0, r1 = K >= 2 ? 2 * h + 1 : 0;
        th2[h] = kDwt ? p_pack(thc[r0], thc[r1]) : 0ull;
        tk2[h] = kDwt ? p_pack(thc2[r0], thc2[r1]) : 0ull;
        st2[h] = kDwt ? p_pack(stp_[r0], stp_[r1]) : 0ull;
    }
    // H words at a time: one slot (K >= 2) or two slots (K = 1); an odd n
    // with K = 1 leaves one scalar
    const int groups = K >= 2 ? n : (n >> 1);
    const uint32_t xb = (uint32_t)__cvta_generic_to_shared(xs);
    for (int q = threadIdx.x; q < groups; q += blockDim.x) {
        f32x2 x[H];
        lds_p<2 * H>(xb + (uint32_t)q * 8 * H, x);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            if constexpr (kDwt) dwt_x2(x[h], th2[h], tk2[h], st2[h]);
            if constexpr (kWrap) x[h] = p_wrap(x[h]);
        }
        sts_p<2 * H>(xb + (uint32_t)q * 8 * H, x);
    }
    if (K == 1 && (n & 1) && threadIdx.x == 0) {
        float x[1] = {xs[n - 1]};
        if (kDwt && in_windows(x[0], thc[0], thc2[0])) x[0] = __fadd_rn(x[0], stp_[0]);
        if (kWrap) x[0] = wrap_c(x[0]);
        xs[n - 1] = x[0];
    }
}

// ---------------------------------------------------------------- paired 16-bit lattice
// Lattice passes of 16-bit storage (binary16, bfloat16) in f32x2 lanes: a
// storage word holds two replicas of a slot, which become one f32x2 pair;
// the two colours of a pass update it as the binary32 passes do, and the
// store wraps it and rounds it to the storage type (round to nearest even),
// exactly as the scalar passes do per lane, so the phases equal theirs bit
// for bit.
// Sign flips of the 16-bit lattice passes on the logic pipe: both lanes for
// binary16, one for bfloat16 (whose widening is already logic work).
template <typename H>
__host__ __device__ constexpr int kAlu16() { return std::is_same<H, __half>::value ? 2 : 1; }

template <typename H>
__device__ __forceinline__ f32x2 h2_to_p(uint32_t w)
{
    const float2 f = h2_to_f2<H>(w);
    return p_pack(f.x, f.y);
}
template <typename H>
__device__ __forceinline__ uint32_t p_to_h2(f32x2 x)
{
    return f2_to_h2<H>(p_lo(x), p_hi(x));
}
template <typename H, int NW>
__device__ __forceinline__ void lds_h(uint32_t a, f32x2 (&x)[NW])
{
    uint32_t w[NW];
    ld_words<NW>(a, w);
#pragma unroll
    for (int i = 0; i < NW; ++i) x[i] = h2_to_p<H>(w[i]);
}
template <typename H, int NW>
__device__ __forceinline__ void sts_h(uint32_t a, const f32x2 (&x)[NW])
{
    uint32_t w[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) w[i] = p_to_h2<H>(x[i]);
    st_words<NW>(a, w);
}
template <typename H, int K>
__device__ __forceinline__ void block_pass_even_h2(H *xs, const uint8_t *wnib, float alpha, int Q)
{
    constexpr int NW = K / 2;          // storage words (replica pairs) per slot
    constexpr uint32_t E = K * 2;      // bytes per slot
    const uint32_t a1 = __float_as_uint(alpha), n1 = a1 ^ 0x80000000u;
    const f32x2 a2 = ((f32x2)a1 << 32) | a1, n2 = ((f32x2)n1 << 32) | n1;
    const uint32_t qb = (uint32_t)Q * E, qb2 = 2 * qb, qb3 = 3 * qb, step = blockDim.x * E;
    uint32_t ad = (uint32_t)__cvta_generic_to_shared(xs) + threadIdx.x * E;
    for (int f = threadIdx.x; f < Q; f += blockDim.x, ad += step) {
        const uint32_t wb = __ldg(wnib + f);
        f32x2 xa[NW], xb[NW], xc[NW], xd[NW];
        lds_h<H, NW>(ad, xa);
        lds_h<H, NW>(ad + qb, xb);
        lds_h<H, NW>(ad + qb2, xc);
        lds_h<H, NW>(ad + qb3, xd);
        const f32x2 w0 = (wb & 1u) ? n2 : a2, w1 = (wb & 2u) ? n2 : a2;
        const f32x2 w2 = (wb & 4u) ? n2 : a2, w3 = (wb & 8u) ? n2 : a2;
#pragma unroll
        for (int h = 0; h < NW; ++h) {
            pair_x2<kAlu16<H>()>(xa[h], xb[h], w0, kTwo2);
            pair_x2<kAlu16<H>()>(xc[h], xd[h], w1, kTwo2);
            pair_x2<kAlu16<H>()>(xa[h], xc[h], w2, kTwo2);
            pair_x2<kAlu16<H>()>(xb[h], xd[h], w3, kTwo2);
            xa[h] = p_wrap(xa[h]);
            xb[h] = p_wrap(xb[h]);
            xc[h] = p_wrap(xc[h]);
            xd[h] = p_wrap(xd[h]);
        }
        sts_h<H, NW>(ad, xa);
        sts_h<H, NW>(ad + qb, xb);
        sts_h<H, NW>(ad + qb2, xc);
        sts_h<H, NW>(ad + qb3, xd);
    }
}

template <typename H, int K, bool kRowWrap, bool kDwt>
__device__ __forceinline__ void odd_block_h2(uint32_t ad, uint32_t oC, uint32_t oB, uint32_t oA, uint32_t wb,
                                             uint32_t a1, f32x2 tzc, const f32x2 (&th2)[K / 2],
                                             const f32x2 (&tk2)[K / 2], const f32x2 (&st2)[K / 2])
{
    constexpr int NW = K / 2;
    constexpr f32x2 tzr = kRowWrap ? kMinusTwo2 : kTwo2;
    const uint32_t n1 = a1 ^ 0x80000000u;
    const f32x2 a2 = ((f32x2)a1 << 32) | a1, n2 = ((f32x2)n1 << 32) | n1;
    f32x2 xd[NW], xc[NW], xb[NW], xa[NW];
    lds_h<H, NW>(ad, xd);
    lds_h<H, NW>(ad + oC, xc);
    lds_h<H, NW>(ad + oB, xb);
    lds_h<H, NW>(ad + oA, xa);
    const f32x2 w0 = (wb & 1u) ? n2 : a2, w1 = (wb & 2u) ? n2 : a2;
    const f32x2 w2 = (wb & 4u) ? n2 : a2, w3 = (wb & 8u) ? n2 : a2;
#pragma unroll
    for (int h = 0; h < NW; ++h) {
        // colour 2: D-C, B-A; colour 3: D-B, C-A
        pair_x2<kAlu16<H>()>(xd[h], xc[h], w0, tzc);
        pair_x2<kAlu16<H>()>(xb[h], xa[h], w1, tzc);
        pair_x2<kAlu16<H>()>(xd[h], xb[h], w2, tzr);
        pair_x2<kAlu16<H>()>(xc[h], xa[h], w3, tzr);
        if constexpr (kDwt) {
            // the twist follows the last colour, before the store rounds
            dwt_x2(xd[h], th2[h], tk2[h], st2[h]);
            dwt_x2(xc[h], th2[h], tk2[h], st2[h]);
            dwt_x2(xb[h], th2[h], tk2[h], st2[h]);
            dwt_x2(xa[h], th2[h], tk2[h], st2[h]);
        }
        xd[h] = p_wrap(xd[h]);
        xc[h] = p_wrap(xc[h]);
        xb[h] = p_wrap(xb[h]);
        xa[h] = p_wrap(xa[h]);
    }
    sts_h<H, NW>(ad, xd);
    sts_h<H, NW>(ad + oC, xc);
    sts_h<H, NW>(ad + oB, xb);
    sts_h<H, NW>(ad + oA, xa);
}

template <typename H, int K, bool kFixedColumn, bool kDwt>
__device__ __forceinline__ void block_pass_odd_h2(H *xs, const uint8_t *wnib, float alpha, int Q, int Wd, int m0,
                                                  int dm, const float *thc, const float *thc2, const float *stp_)
{
    constexpr uint32_t E = K * 2;  // bytes per slot
    const uint32_t a1 = __float_as_uint(alpha);
    f32x2 th2[K / 2], tk2[K / 2], st2[K / 2];
#pragma unroll
    for (int h = 0; h < K / 2; ++h) {
        th2[h] = kDwt ? p_pack(thc[2 * h], thc[2 * h + 1]) : 0ull;
        tk2[h] = kDwt ? p_pack(thc2[2 * h], thc2[2 * h + 1]) : 0ull;
        st2[h] = kDwt ? p_pack(stp_[2 * h], stp_[2 * h + 1]) : 0ull;
    }
    const uint32_t qb = (uint32_t)Q * E;
    const uint32_t wdb = (uint32_t)Wd * E;
    const uint32_t rowwrap = (uint32_t)(Wd - Q) * E;
    const uint32_t step = blockDim.x * E;
    uint32_t ad = (uint32_t)__cvta_generic_to_shared(xs) + 3 * qb + threadIdx.x * E;
    int m = m0;
    bool cw = (m0 == Wd - 1);
    uint32_t goffb = cw ? (uint32_t)(1 - Wd) * E : E;
    const int qlast = Q - Wd;
    int f = threadIdx.x;
#pragma unroll 4
    for (; f < qlast; f += blockDim.x, ad += step) {
        if (!kFixedColumn) {
            cw = (m == Wd - 1);
            goffb = cw ? (uint32_t)(1 - Wd) * E : E;
            m += dm;
            if (m >= Wd) m -= Wd;
        }
        const uint32_t wb = __ldg(wnib + Q + f) ^ (cw ? 3u : 0u);
        odd_block_h2<H, K, false, kDwt>(ad, goffb - qb, wdb - 2 * qb, goffb + wdb - 3 * qb, wb, a1,
                                        cw ? kMinusTwo2 : kTwo2, th2, tk2, st2);
    }
    for (; f < Q; f += blockDim.x, ad += step) {
        if (!kFixedColumn) {
            cw = (m == Wd - 1);
            goffb = cw ? (uint32_t)(1 - Wd) * E : E;
            m += dm;
            if (m >= Wd) m -= Wd;
        }
        const uint32_t wb = __ldg(wnib + Q + f) ^ (cw ? 3u : 0u) ^ 12u;
        odd_block_h2<H, K, true, kDwt>(ad, goffb - qb, rowwrap - 2 * qb, goffb + rowwrap - 3 * qb, wb, a1,
                                       cw ? kMinusTwo2 : kTwo2, th2, tk2, st2);
    }
}

// 16-bit storage (binary16, bfloat16) on edge lists: one batch of B edges
// per thread, each slot's NW words widened to f32x2 pairs (two replicas a
// pair), eq. (6) as in the binary32 sweep, and every updated phase wrapped
// and rounded to the storage type when stored -- after every update, as
// the oracle's per-update rounding for edge lists has it. kTail and kSgn as
// in edge_batch_x2.
template <typename H, int NW, int B, bool kTail, bool kSgn>
__device__ __forceinline__ void edge_batch_h2(const InstView &a, uint32_t xb, float alpha, int e0, int e1, int nt)
{
    constexpr uint32_t E = NW * 4;  // bytes per slot
    uint32_t ai[B], aj[B];
    float aw[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int e = e0 + u * nt;
        uint32_t rec = 0;
        int w = 0;
        if (!kTail || e < e1) {
            if constexpr (kSgn) {
                rec = load_rec_sgn(a, e);
            } else {
                rec = load_rec(a, e);
                w = __ldg(a.w + e);
            }
        }
        aj[u] = xb + (rec >> 16) * E;
        if constexpr (kSgn) {
            ai[u] = xb + (rec & 0xFFFEu) * (E / 2);
            aw[u] = __uint_as_float(flip_if_odd(__float_as_uint(alpha), rec));
        } else {
            ai[u] = xb + (rec & 0xFFFFu) * E;
            aw[u] = alpha * weight_f((int8_t)w);
        }
    }
    f32x2 xi[B][NW], xj[B][NW];
#pragma unroll
    for (int u = 0; u < B; ++u) {
        lds_h<H, NW>(ai[u], xi[u]);
        lds_h<H, NW>(aj[u], xj[u]);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const f32x2 aw2 = p_pack(aw[u], aw[u]);
#pragma unroll
        for (int h = 0; h < NW; ++h) {
            pair_x2<kAlu16<H>()>(xi[u][h], xj[u][h], aw2, kTwo2);
            xi[u][h] = p_wrap(xi[u][h]);
            xj[u][h] = p_wrap(xj[u][h]);
        }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
        if (!kTail || e0 + u * nt < e1) {
            sts_h<H, NW>(ai[u], xi[u]);
            sts_h<H, NW>(aj[u], xj[u]);
        }
    }
}

// The colours of one sweep of a 16-bit edge-list tile: whole batches
// without bounds checks, then at most one checked batch per thread.
template <typename H, int K, bool kSgn>
__device__ __forceinline__ void general_colours_h2(const InstView &a, H *xs, float alpha)
{
    constexpr int NW = K / 2, B = K == 8 ? 2 : 3;
    const int nt = blockDim.x;
    const uint32_t xb = (uint32_t)__cvta_generic_to_shared(xs);
    for (int c = 0; c < a.C; ++c) {
        const int e1 = __ldg(a.off + c + 1);
        int e0 = __ldg(a.off + c) + threadIdx.x;
        for (; e0 + (B - 1) * nt < e1; e0 += B * nt) edge_batch_h2<H, NW, B, false, kSgn>(a, xb, alpha, e0, e1, nt);
        if (e0 < e1) edge_batch_h2<H, NW, B, true, kSgn>(a, xb, alpha, e0, e1, nt);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- fixed point sweep
// Eq. (6) on the 2^-16-turn grid: with a phase held as q << 16, d = x_i - x_j
// read as int32 is the minimum angular difference (times 2^32) and the
// biased sign of eq. (4) is d >= 0 (d = -2^31, exactly opposite, gives -1);
// the step is (alpha quanta x w) << 16 and every operation is exact. The
// dual window twist moves a phase iff ((q << 16) + c) mod 2^31 < QW, with
// c = QW/2 - q_theta per replica (2^-32 turn).

// Fixed-point phases stay packed in the sweeps below: a 32-bit word holds
// the u16 phases of replicas 2h (low half) and 2h + 1 (high half) of a
// slot, and add.u16x2 adds per half modulo 2^16, which is the grid's
// circle arithmetic -- the same values as the q << 16 form, without
// widening and packing each phase. Per half, x_j + ~x_i =
// ~(x_i - x_j), whose sign bit is the complement of the sign bit that
// decides eq. (4) (ties and the exactly-opposite value included), and prmt
// replicates each half's sign bit over the half.
__device__ __forceinline__ uint32_t add_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("add.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t half_signs(uint32_t v)
{
    uint32_t m;
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(m) : "r"(v));
    return m;
}
// The low 16 bits of v in both halves.
__device__ __forceinline__ uint32_t both_halves(uint32_t v) { return __byte_perm(v, 0u, 0x1010); }

// Eq. (6) on NW packed words of x_i and x_j: pw is the step alpha w (grid
// quanta) in both halves, nw its negation; x_i gains pw where x_i - x_j >= 0
// and nw elsewhere, x_j the opposite.
template <int NW>
__device__ __forceinline__ void pair_qw(uint32_t (&xi)[NW], uint32_t (&xj)[NW], uint32_t pw, uint32_t nw)
{
#pragma unroll
    for (int h = 0; h < NW; ++h) {
        const uint32_t ge = half_signs(add_u16x2(xj[h], ~xi[h]));
        xi[h] = add_u16x2(xi[h], (pw & ge) | (nw & ~ge));
        xj[h] = add_u16x2(xj[h], (nw & ge) | (pw & ~ge));
    }
}

// The dual window twist on a packed word. With c = ch 2^16 + cl
// (cl < 2^16), ((q << 16) + c) mod 2^31 = ((q + ch) mod 2^15) 2^16 + cl, so
// the test against QW is (q + ch) mod 2^15 < T with T = ceil((QW - cl) /
// 2^16) (0 when QW <= cl): per half, the sign of (q + ch) mod 2^15 - T.
// chw, ntw (= -T), sqw: ch, -T and the step of the word's two replicas.
__device__ __forceinline__ void dwt_qw(uint32_t &x, uint32_t chw, uint32_t ntw, uint32_t sqw)
{
    const uint32_t y = add_u16x2(x, chw) & 0x7FFF7FFFu;
    x = add_u16x2(x, sqw & half_signs(add_u16x2(y, ntw)));
}

// chw, ntw, sqw of the words of a tile from the per-replica c (QW/2 minus
// the window centre, 2^-32 turn), QW and the steps sq (q << 16 form).
template <int NW>
__device__ __forceinline__ void dwt_qw_consts(const uint32_t *c, uint32_t qw, const uint32_t *sq, uint32_t (&chw)[NW],
                                              uint32_t (&ntw)[NW], uint32_t (&sqw)[NW])
{
#pragma unroll
    for (int h = 0; h < NW; ++h) {
        uint32_t nt[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint32_t cl = c[2 * h + k] & 0xFFFFu;
            const uint32_t T = qw > cl ? (qw - cl + 0xFFFFu) >> 16 : 0u;
            nt[k] = (0u - T) & 0xFFFFu;
        }
        chw[h] = __byte_perm(c[2 * h], c[2 * h + 1], 0x7632);
        ntw[h] = nt[0] | (nt[1] << 16);
        sqw[h] = __byte_perm(sq[2 * h], sq[2 * h + 1], 0x7632);
    }
}

// NW packed words of a slot at a 32-bit shared address.
template <int NW>
__device__ __forceinline__ void lds_w(uint32_t a, uint32_t (&x)[NW])
{
    if constexpr (NW == 1) {
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(x[0]) : "r"(a) : "memory");
    } else if constexpr (NW == 2) {
        asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(x[0]), "=r"(x[1]) : "r"(a) : "memory");
    } else {
        static_assert(NW == 4, "NW");
        asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]) : "r"(a) : "memory");
    }
}
template <int NW>
__device__ __forceinline__ void sts_w(uint32_t a, const uint32_t (&x)[NW])
{
    if constexpr (NW == 1) {
        asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(x[0]) : "memory");
    } else if constexpr (NW == 2) {
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(x[0]), "r"(x[1]) : "memory");
    } else {
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x[0]), "r"(x[1]), "r"(x[2]),
                     "r"(x[3]) : "memory");
    }
}

// One batch of B edges per thread of the edge-list sweep on packed words
// (edges e0, e0 + nt, ...); kTail: the batch may run past the end e1 of its
// colour (its loads and stores skipped there); kSgn: the records of a.ijs,
// whose bit 0 is the sign of a +-1 weight (no weight load).
template <int NW, int B, bool kTail, bool kSgn>
__device__ __forceinline__ void edge_batch_qw(const InstView &a, uint32_t xb, uint32_t aq, int e0, int e1, int nt)
{
    constexpr uint32_t E = NW * 4;  // bytes per slot
    uint32_t ai[B], aj[B], pw[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int e = e0 + u * nt;
        uint32_t rec = 0u;
        int32_t w = 0;
        if (!kTail || e < e1) {
            if constexpr (kSgn) {
                rec = load_rec_sgn(a, e);
            } else {
                rec = load_rec(a, e);
                w = (int32_t)__ldg(a.w + e);
            }
        }
        aj[u] = xb + (rec >> 16) * E;
        if constexpr (kSgn) {
            ai[u] = xb + (rec & 0xFFFEu) * (E / 2);
            pw[u] = (rec & 1u) ? 0u - aq : aq;
        } else {
            ai[u] = xb + (rec & 0xFFFFu) * E;
            pw[u] = (uint32_t)((int32_t)aq * w);
        }
    }
    uint32_t xi[B][NW], xj[B][NW];
#pragma unroll
    for (int u = 0; u < B; ++u) {
        if (!kTail || e0 + u * nt < e1) {
            lds_w<NW>(ai[u], xi[u]);
            lds_w<NW>(aj[u], xj[u]);
        } else {
#pragma unroll
            for (int h = 0; h < NW; ++h) xi[u][h] = xj[u][h] = 0u;
        }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) pair_qw<NW>(xi[u], xj[u], both_halves(pw[u]), both_halves(0u - pw[u]));
#pragma unroll
    for (int u = 0; u < B; ++u) {
        if (!kTail || e0 + u * nt < e1) {
            sts_w<NW>(ai[u], xi[u]);
            sts_w<NW>(aj[u], xj[u]);
        }
    }
}

// One colour of the edge-list sweep on packed words: whole batches without
// bounds checks, then at most one checked batch per thread.
template <int K>
__device__ __forceinline__ void general_colour_qw(const InstView &a, uint16_t *xs, int c, uint32_t aq)
{
    // 3 edges per thread for tiles of 2 or 4 replicas, 2 for tiles of 8, so
    // that 1,024 threads fit the 64-register cap
    constexpr int NW = K / 2, B = K == 8 ? 2 : 3;
    const int nt = blockDim.x;
    const uint32_t xb = (uint32_t)__cvta_generic_to_shared(xs);
    const int e1 = __ldg(a.off + c + 1);
    int e0 = __ldg(a.off + c) + threadIdx.x;
    if (a.ijs) {
        for (; e0 + (B - 1) * nt < e1; e0 += B * nt) edge_batch_qw<NW, B, false, true>(a, xb, aq, e0, e1, nt);
        if (e0 < e1) edge_batch_qw<NW, B, true, true>(a, xb, aq, e0, e1, nt);
    } else {
        for (; e0 + (B - 1) * nt < e1; e0 += B * nt) edge_batch_qw<NW, B, false, false>(a, xb, aq, e0, e1, nt);
        if (e0 < e1) edge_batch_qw<NW, B, true, false>(a, xb, aq, e0, e1, nt);
    }
}

// The lattice passes of the fixed-point sweep on packed words (the 2x2
// blocks of block_pass_even / block_pass_odd). pw, nw: alpha quanta and
// their negation in both halves; a set weight bit (w = -1) swaps them.
template <int K>
__device__ __forceinline__ void block_pass_even_qw(uint16_t *xs, const uint8_t *wnib, uint32_t pw, uint32_t nw, int Q)
{
    constexpr int NW = K / 2;
    constexpr uint32_t E = K * 2;  // bytes per slot
    const uint32_t qb = (uint32_t)Q * E, qb2 = 2 * qb, qb3 = 3 * qb, step = blockDim.x * E;
    uint32_t ad = (uint32_t)__cvta_generic_to_shared(xs) + threadIdx.x * E;
    for (int f = threadIdx.x; f < Q; f += blockDim.x, ad += step) {
        const uint32_t wb = __ldg(wnib + f);
        uint32_t xa[NW], xb[NW], xc[NW], xd[NW];
        lds_w<NW>(ad, xa);
        lds_w<NW>(ad + qb, xb);
        lds_w<NW>(ad + qb2, xc);
        lds_w<NW>(ad + qb3, xd);
        pair_qw<NW>(xa, xb, (wb & 1u) ? nw : pw, (wb & 1u) ? pw : nw);
        pair_qw<NW>(xc, xd, (wb & 2u) ? nw : pw, (wb & 2u) ? pw : nw);
        pair_qw<NW>(xa, xc, (wb & 4u) ? nw : pw, (wb & 4u) ? pw : nw);
        pair_qw<NW>(xb, xd, (wb & 8u) ? nw : pw, (wb & 8u) ? pw : nw);
        sts_w<NW>(ad, xa);
        sts_w<NW>(ad + qb, xb);
        sts_w<NW>(ad + qb2, xc);
        sts_w<NW>(ad + qb3, xd);
    }
}

// In the shifted blocks the second slot holds the smaller original id at a
// torus wrap; the roles of eq. (6) then swap exactly (the exactly-opposite
// tie is an integer value on the grid, so no shortcut is taken).
template <int NW>
__device__ __forceinline__ void pair_qw_oriented(uint32_t (&x1)[NW], uint32_t (&x2)[NW], uint32_t pw, uint32_t nw,
                                                 bool swp)
{
    if (swp) pair_qw<NW>(x2, x1, pw, nw);
    else pair_qw<NW>(x1, x2, pw, nw);
}

template <int K, bool kFixedColumn>
__device__ __forceinline__ void block_pass_odd_qw(uint16_t *xs, const uint8_t *wnib, uint32_t pw, uint32_t nw, int Q,
                                                  int Wd, int m0, int dm, bool dwt, const uint32_t *c, uint32_t qw,
                                                  const uint32_t *sqs)
{
    constexpr int NW = K / 2;
    constexpr uint32_t E = K * 2;  // bytes per slot
    uint32_t chw[NW], ntw[NW], sqw[NW];  // the twist's constants per word (steps 0 off the DWT sweeps)
    if (dwt) {
        dwt_qw_consts<NW>(c, qw, sqs, chw, ntw, sqw);
    } else {
#pragma unroll
        for (int h = 0; h < NW; ++h) chw[h] = ntw[h] = sqw[h] = 0u;
    }
    // byte offsets from D[f] to C[g], B[h], A[gh] (g: next column, h: next row)
    const uint32_t qb = (uint32_t)Q * E, wdb = (uint32_t)Wd * E, rowwrap = (uint32_t)(Wd - Q) * E;
    const uint32_t step = blockDim.x * E;
    uint32_t ad = (uint32_t)__cvta_generic_to_shared(xs) + 3 * qb + threadIdx.x * E;
    int m = m0;
    const bool cw0 = (m0 == Wd - 1);
    const uint32_t goffb0 = cw0 ? (uint32_t)(1 - Wd) * E : E;
    for (int f = threadIdx.x; f < Q; f += blockDim.x, ad += step) {
        uint32_t goffb = goffb0;
        bool cw = cw0;
        if (!kFixedColumn) {
            cw = (m == Wd - 1);
            goffb = cw ? (uint32_t)(1 - Wd) * E : E;
            m += dm;
            if (m >= Wd) m -= Wd;
        }
        const bool rw = (f >= Q - Wd);
        const uint32_t hoffb = rw ? rowwrap : wdb;
        const uint32_t aC = ad - qb + goffb, aB = ad - 2 * qb + hoffb, aA = ad - 3 * qb + goffb + hoffb;
        const uint32_t wb = __ldg(wnib + Q + f);
        uint32_t xd[NW], xc[NW], xb[NW], xa[NW];
        lds_w<NW>(ad, xd);
        lds_w<NW>(aC, xc);
        lds_w<NW>(aB, xb);
        lds_w<NW>(aA, xa);
        pair_qw_oriented<NW>(xd, xc, (wb & 1u) ? nw : pw, (wb & 1u) ? pw : nw, cw);
        pair_qw_oriented<NW>(xb, xa, (wb & 2u) ? nw : pw, (wb & 2u) ? pw : nw, cw);
        pair_qw_oriented<NW>(xd, xb, (wb & 4u) ? nw : pw, (wb & 4u) ? pw : nw, rw);
        pair_qw_oriented<NW>(xc, xa, (wb & 8u) ? nw : pw, (wb & 8u) ? pw : nw, rw);
        if (dwt) {
#pragma unroll
            for (int h = 0; h < NW; ++h) {
                dwt_qw(xd[h], chw[h], ntw[h], sqw[h]);
                dwt_qw(xc[h], chw[h], ntw[h], sqw[h]);
                dwt_qw(xb[h], chw[h], ntw[h], sqw[h]);
                dwt_qw(xa[h], chw[h], ntw[h], sqw[h]);
            }
        }
        sts_w<NW>(ad, xd);
        sts_w<NW>(aC, xc);
        sts_w<NW>(aB, xb);
        sts_w<NW>(aA, xa);
    }
}

// ---------------------------------------------------------------- segment body
enum { MODE_GENERAL = 0, MODE_ACCUM = 1, MODE_LATTICE2D = 2 };

// Local fields (eq. (1)) as couplings J = h to a reference phase frozen at
// 0: eq. (6) on x_v alone with x_j = 0, i.e. the step alpha (-h) s with
// s = +1 iff the minimum angular difference of x_v from 0 is >= 0. Each
// vertex appears once, so the field updates form one more conflict-free
// sub-sweep, after the colours.
template <typename Store, int K>
__device__ __forceinline__ void field_pass(const InstView &a, Store *xs, float alpha)
{
    for (int u = threadIdx.x; u < a.n; u += blockDim.x) {
        const int hvu = __ldg(a.hv + u);
        if (hvu == 0) continue;
        const float aw = alpha * (float)(-hvu);
        float x[K];
        ldk<K>(xs + (size_t)u * K, x);
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const float st = floor_parity(2.0f, x[r]) ? -aw : aw;
            x[r] = wrap_c(__fadd_rn(x[r], st));
        }
        stk<K>(xs + (size_t)u * K, x);
    }
}

template <int K>
__device__ __forceinline__ void field_pass_q(const InstView &a, uint16_t *xs, uint32_t aq)
{
    for (int u = threadIdx.x; u < a.n; u += blockDim.x) {
        const int hvu = __ldg(a.hv + u);
        if (hvu == 0) continue;
        const uint32_t ap = (aq * (uint32_t)(-hvu)) << 16;
        uint32_t x[K];
        ldq<K>(xs + (size_t)u * K, x);
#pragma unroll
        for (int r = 0; r < K; ++r) x[r] += ((int32_t)x[r] >= 0) ? ap : 0u - ap;
        stq<K>(xs + (size_t)u * K, x);
    }
}

// True after the sweeps at which a tracking readout is due.
__device__ __forceinline__ bool readout_due(const InstView &v, int64_t s)
{
    return v.track > 0 && (s % v.track == 0 || s == v.S);
}

// Fixed-point (COSM_Q16) segment: as run_segment below, on the grid.
template <int K, int kMode>
__device__ __forceinline__ void run_segment_q16(const InstView &v, const Segment &sg, unsigned char *smem,
                                                int *s_skip, int32_t *ready, int32_t *err,
                                                uint64_t wait_limit_ns)
{
    const Tile<uint16_t, K> t = carve<uint16_t, K>(smem, v.n, v.P, kMode == MODE_ACCUM);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = v.n;
    const bool dwt_on = !(v.flags & COSM_NO_DWT) && v.dwt_period > 0;
    const bool randdir = (v.flags & COSM_DWT_RANDOM_DIR) != 0;
    uint32_t *cq = reinterpret_cast<uint32_t *>(t.thc);
    uint32_t *sqs = reinterpret_cast<uint32_t *>(t.stp);
    int m0 = 0, dm = 0;
    if (kMode == MODE_LATTICE2D) {
        m0 = tid % v.Wd;
        dm = nt % v.Wd;
    }
    if (!seg_begin<uint16_t, K>(v, sg, t, s_skip, ready, err, wait_limit_ns)) return;
    const uint32_t rep0 = (uint32_t)sg.tile * K;
    int phase = dwt_on ? (int)(sg.s_begin % v.dwt_period) : 1;
    for (int64_t s = sg.s_begin; s <= sg.s_end; ++s) {
        const float2 at = __ldg(v.alpha_tab + (s - v.alpha_base));  // grid quanta
        const uint32_t aq = (uint32_t)__float2int_rn(at.x), stepq = (uint32_t)__float2int_rn(at.y) << 16;
        const bool dwt = dwt_on && phase == 0;
        if (dwt && tid < K) {
            bool neg = false;
            const uint32_t qth = (uint32_t)__float2uint_rn(dwt_theta(v.seed, rep0 + tid, s, &neg) * 16777216.0f) << 8;
            cq[tid] = (v.qwin >> 1) - qth;
            sqs[tid] = (randdir && neg) ? 0u - stepq : stepq;
        }
        if (kMode == MODE_LATTICE2D) {
            const uint32_t pw = both_halves(aq), nw = both_halves(0u - aq);
            block_pass_even_qw<K>(t.xs, v.wnib, pw, nw, v.Q);
            __syncthreads();
            if (dm == 0)
                block_pass_odd_qw<K, true>(t.xs, v.wnib, pw, nw, v.Q, v.Wd, m0, dm, dwt, cq, v.qwin, sqs);
            else
                block_pass_odd_qw<K, false>(t.xs, v.wnib, pw, nw, v.Q, v.Wd, m0, dm, dwt, cq, v.qwin, sqs);
            __syncthreads();
        } else {
            if (kMode == MODE_GENERAL) {
                for (int c = 0; c < v.C; ++c) {
                    general_colour_qw<K>(v, t.xs, c, aq);
                    __syncthreads();
                }
                if (v.hv) {
                    field_pass_q<K>(v, t.xs, aq);
                    __syncthreads();
                }
            } else {
                // simultaneous step (eq. (8)): integer sums of the pair steps
                uint32_t *acc = reinterpret_cast<uint32_t *>(t.acc);
                for (int k = tid; k < n * K; k += nt) acc[k] = 0u;
                __syncthreads();
                for (int c = 0; c < v.C; ++c) {
                    const int e1 = __ldg(v.off + c + 1);
                    for (int e = __ldg(v.off + c) + tid; e < e1; e += nt) {
                        const uint32_t rec = load_rec(v, e);
                        const uint32_t ap = (uint32_t)((int32_t)aq * (int32_t)__ldg(v.w + e)) << 16;
                        const int i = (int)(rec & 0xFFFFu), j = (int)(rec >> 16);
                        uint32_t xi[K], xj[K];
                        ldq<K>(t.xs + (size_t)i * K, xi);
                        ldq<K>(t.xs + (size_t)j * K, xj);
#pragma unroll
                        for (int r = 0; r < K; ++r) {
                            const uint32_t st = ((int32_t)(xi[r] - xj[r]) >= 0) ? ap : 0u - ap;
                            acc[(size_t)i * K + r] += st;
                            acc[(size_t)j * K + r] -= st;
                        }
                    }
                    __syncthreads();
                }
                for (int u = tid; u < n; u += nt) {
                    uint32_t x[K];
                    ldq<K>(t.xs + (size_t)u * K, x);
                    const int hvu = v.hv ? __ldg(v.hv + u) : 0;
                    const uint32_t ap = (aq * (uint32_t)(-hvu)) << 16;
#pragma unroll
                    for (int r = 0; r < K; ++r) {
                        const uint32_t fs = hvu ? (((int32_t)x[r] >= 0) ? ap : 0u - ap) : 0u;
                        x[r] += acc[(size_t)u * K + r] + fs;
                    }
                    stq<K>(t.xs + (size_t)u * K, x);
                }
                __syncthreads();
            }
            if (dwt) {
                if (v.C == 0) __syncthreads();
                constexpr int NW = K / 2;
                uint32_t chw[NW], ntw[NW], sqw[NW];
                dwt_qw_consts<NW>(cq, v.qwin, sqs, chw, ntw, sqw);
                const uint32_t xb = (uint32_t)__cvta_generic_to_shared(t.xs);
                for (int u = tid; u < n; u += nt) {
                    uint32_t x[NW];
                    lds_w<NW>(xb + (uint32_t)u * (K * 2), x);
#pragma unroll
                    for (int h = 0; h < NW; ++h) dwt_qw(x[h], chw[h], ntw[h], sqw[h]);
                    sts_w<NW>(xb + (uint32_t)u * (K * 2), x);
                }
                __syncthreads();
            }
        }
        if (readout_due(v, s)) tile_readout<uint16_t, K>(v, sg.tile, t, (int)((s - 1) / v.track), true);
        if (dwt_on && ++phase == v.dwt_period) phase = 0;
    }
    seg_end<uint16_t, K>(v, sg, t, ready);
}

// One work segment of one replica tile: wait / init / load, sweeps
// s_begin..s_end, readout, store / publish. Every thread of the CTA calls it.
template <typename Store, int K, int kMode>
__device__ __forceinline__ void run_segment_fp(const InstView &v, const Segment &sg, unsigned char *smem,
                                               int *s_skip, int32_t *ready, int32_t *err,
                                               uint64_t wait_limit_ns)
{
    const Tile<Store, K> t = carve<Store, K>(smem, v.n, v.P, kMode == MODE_ACCUM);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = v.n;
    const bool dwt_on = !(v.flags & COSM_NO_DWT) && v.dwt_period > 0;
    const bool randdir = (v.flags & COSM_DWT_RANDOM_DIR) != 0;
    const float W2 = 2.0f * v.window, hw = 0.5f * v.window;
    constexpr bool kLattice = (kMode == MODE_LATTICE2D);
    int m0 = 0, dm = 0;
    if (kLattice) {
        m0 = tid % v.Wd;
        dm = nt % v.Wd;
    }
    if (!seg_begin<Store, K>(v, sg, t, s_skip, ready, err, wait_limit_ns)) return;
    const uint32_t rep0 = (uint32_t)sg.tile * K;
    int phase = dwt_on ? (int)(sg.s_begin % v.dwt_period) : 1;
    int stage_cur = 0;  // staged edge records: the buffer holding colour 0
    for (int64_t s = sg.s_begin; s <= sg.s_end; ++s) {
        const float2 at = __ldg(v.alpha_tab + (s - v.alpha_base));
        const bool dwt = dwt_on && phase == 0;
        // binary32 lattice phases are wrapped on every wrap_p-th sweep of the
        // trial (16-bit storage: every sweep)
        const bool wrap = sizeof(Store) == 2 || v.wrap_p <= 1 || (s % v.wrap_p) == 0;
        if (dwt && tid < K) {
            bool neg = false;
            const float c = 2.0f * (hw - dwt_theta(v.seed, rep0 + tid, s, &neg));
            t.thc[tid] = c;
            t.thc2[tid] = c - W2;
            t.stp[tid] = (randdir && neg) ? -at.y : at.y;
        }
        if (kLattice) {
            // colours 0, 1 in the 2x2 blocks; colours 2, 3 (+ DWT) in the
            // shifted blocks; binary32 tiles of an even width in f32x2 pairs
            constexpr bool kPaired = sizeof(Store) == 4 && (K == 2 || K == 4);
            if (K == 2 && kPaired && v.paired == 2) {
                if constexpr (K == 2 && kPaired) {
                    float *xf = reinterpret_cast<float *>(t.xs);
                    block_pass_even_x2p(xf, v.wnib, at.x, v.Q);
                    __syncthreads();
                    if (dm == 0)
                        block_pass_odd_x2_sel<K, true>(xf, v.wnib, at.x, v.Q, v.Wd, m0, dm, dwt, wrap, t.thc, t.thc2,
                                                       t.stp);
                    else
                        block_pass_odd_x2_sel<K, false>(xf, v.wnib, at.x, v.Q, v.Wd, m0, dm, dwt, wrap, t.thc, t.thc2,
                                                        t.stp);
                    __syncthreads();
                }
            } else if (kPaired && v.paired) {
                if constexpr (kPaired) {
                    float *xf = reinterpret_cast<float *>(t.xs);
                    block_pass_even_x2<K>(xf, v.wnib, at.x, v.Q);
                    __syncthreads();
                    if (dm == 0)
                        block_pass_odd_x2_sel<K, true>(xf, v.wnib, at.x, v.Q, v.Wd, m0, dm, dwt, wrap, t.thc, t.thc2,
                                                       t.stp);
                    else
                        block_pass_odd_x2_sel<K, false>(xf, v.wnib, at.x, v.Q, v.Wd, m0, dm, dwt, wrap, t.thc, t.thc2,
                                                        t.stp);
                    __syncthreads();
                }
            } else if (sizeof(Store) == 2 && v.paired) {
                // 16-bit storage: f32x2 lanes over the replica pairs of a word
                if constexpr (sizeof(Store) == 2) {
                    block_pass_even_h2<Store, K>(t.xs, v.wnib, at.x, v.Q);
                    __syncthreads();
                    if (dm == 0) {
                        if (dwt)
                            block_pass_odd_h2<Store, K, true, true>(t.xs, v.wnib, at.x, v.Q, v.Wd, m0, dm, t.thc,
                                                                    t.thc2, t.stp);
                        else
                            block_pass_odd_h2<Store, K, true, false>(t.xs, v.wnib, at.x, v.Q, v.Wd, m0, dm, t.thc,
                                                                     t.thc2, t.stp);
                    } else {
                        if (dwt)
                            block_pass_odd_h2<Store, K, false, true>(t.xs, v.wnib, at.x, v.Q, v.Wd, m0, dm, t.thc,
                                                                     t.thc2, t.stp);
                        else
                            block_pass_odd_h2<Store, K, false, false>(t.xs, v.wnib, at.x, v.Q, v.Wd, m0, dm, t.thc,
                                                                      t.thc2, t.stp);
                    }
                    __syncthreads();
                }
            } else {
                block_pass_even<Store, K>(t.xs, v.wnib, at.x, v.Q);
                __syncthreads();
                if (wrap) {
                    if (dm == 0)
                        block_pass_odd<Store, K, true, true>(t.xs, v.wnib, at.x, v.Q, v.Wd, m0, dm, dwt, t.thc, t.thc2,
                                                             t.stp);
                    else
                        block_pass_odd<Store, K, false, true>(t.xs, v.wnib, at.x, v.Q, v.Wd, m0, dm, dwt, t.thc,
                                                              t.thc2, t.stp);
                } else if constexpr (sizeof(Store) == 4) {
                    if (dm == 0)
                        block_pass_odd<Store, K, true, false>(t.xs, v.wnib, at.x, v.Q, v.Wd, m0, dm, dwt, t.thc,
                                                              t.thc2, t.stp);
                    else
                        block_pass_odd<Store, K, false, false>(t.xs, v.wnib, at.x, v.Q, v.Wd, m0, dm, dwt, t.thc,
                                                               t.thc2, t.stp);
                }
                __syncthreads();
            }
        } else {
            if (kMode == MODE_GENERAL) {
                // sequential conflict-free search: colours in order (eq. (11))
                if constexpr (sizeof(Store) == 4) {
                    static_assert(K == 1 || K == 2 || K == 4, "binary32 tiles hold 1, 2 or 4 replicas");
                    // binary32: f32x2 lanes (replica pairs, or edge pairs for
                    // single-replica tiles); batches of 3 edges for tiles of
                    // two replicas (4 and 5 were 1-5 % slower: the last,
                    // checked batch of a colour wastes fewer slots), 2 for
                    // tiles of four (their registers), 4 for one (pairs)
                    float *xf = reinterpret_cast<float *>(t.xs);
                    constexpr int kB = K == 4 ? 2 : (K == 2 ? 3 : 4);
                    if (v.stage_ij) {
                        const uint32_t stage = (uint32_t)__cvta_generic_to_shared(smem) +
                                               (uint32_t)smem_bytes<Store, K>(v.n, v.P, false);
                        const bool first = s == sg.s_begin, last = s == sg.s_end;
                        if (v.wrap_p == 0)
                            general_colours_x2s<K, kB, true>(v, xf, at.x, stage, first, last, stage_cur);
                        else
                            general_colours_x2s<K, kB, false>(v, xf, at.x, stage, first, last, stage_cur);
                    } else if (v.wrap_p == 0) {
                        general_colours_x2<K, kB, true>(v, xf, at.x);
                    } else if (v.ijs) {
                        general_colours_x2<K, kB, false, true>(v, xf, at.x);
                    } else {
                        general_colours_x2<K, kB, false>(v, xf, at.x);
                    }
                } else {
                    // 16-bit storage: f32x2 lanes over the replica pairs of a word
                    if (v.ijs) general_colours_h2<Store, K, true>(v, t.xs, at.x);
                    else general_colours_h2<Store, K, false>(v, t.xs, at.x);
                }
                if (v.hv) {
                    field_pass<Store, K>(v, t.xs, at.x);
                    __syncthreads();
                }
            } else {
                // simultaneous generalized-gradient step over all edges (eq. (8))
                for (int k = tid; k < n * K; k += nt) t.acc[k] = 0.0f;
                __syncthreads();
                for (int c = 0; c < v.C; ++c) {
                    const int e1 = __ldg(v.off + c + 1);
                    for (int e = __ldg(v.off + c) + tid; e < e1; e += nt) {
                        const uint32_t rec = load_rec(v, e);
                        const float aw = at.x * (float)__ldg(v.w + e);
                        const int i = (int)(rec & 0xFFFFu), j = (int)(rec >> 16);
                        float xi[K], xj[K];
                        ldk<K>(t.xs + (size_t)i * K, xi);
                        ldk<K>(t.xs + (size_t)j * K, xj);
#pragma unroll
                        for (int r = 0; r < K; ++r) {
                            const float d = __fadd_rn(xi[r], -xj[r]);
                            const float st = floor_parity(2.0f, d) ? -aw : aw;
                            t.acc[(size_t)i * K + r] += st;
                            t.acc[(size_t)j * K + r] -= st;
                        }
                    }
                    __syncthreads();  // one colour is a matching: no shared vertex
                }
                for (int u = tid; u < n; u += nt) {
                    float x[K];
                    ldk<K>(t.xs + (size_t)u * K, x);
                    const int hvu = v.hv ? __ldg(v.hv + u) : 0;
                    const float aw = at.x * (float)(-hvu);
#pragma unroll
                    for (int r = 0; r < K; ++r) {
                        float dx = t.acc[(size_t)u * K + r];
                        if (hvu) dx = __fadd_rn(dx, floor_parity(2.0f, x[r]) ? -aw : aw);
                        x[r] = wrap_c(__fadd_rn(x[r], dx));
                    }
                    stk<K>(t.xs + (size_t)u * K, x);
                }
                __syncthreads();
            }
            // binary32 edge lists: the twist and the wrap (on every
            // wrap_p-th sweep, or with every twist when each update is
            // wrapped) in one pass of f32x2 words
            constexpr bool kGenF32 = kMode == MODE_GENERAL && sizeof(Store) == 4 && K <= 4;
            const bool wrap_sweep = kGenF32 && (v.wrap_p == 0 ? dwt : (s % v.wrap_p) == 0);
            if (kGenF32 && (dwt || wrap_sweep)) {
                if constexpr (kGenF32) {
                    if (v.C == 0) __syncthreads();
                    float *xf = reinterpret_cast<float *>(t.xs);
                    if (dwt && wrap_sweep) twist_wrap_x2<K, true, true>(xf, n, t.thc, t.thc2, t.stp);
                    else if (dwt) twist_wrap_x2<K, true, false>(xf, n, t.thc, t.thc2, t.stp);
                    else twist_wrap_x2<K, false, true>(xf, n, t.thc, t.thc2, t.stp);
                    __syncthreads();
                }
            } else if (dwt) {
                if (v.C == 0) __syncthreads();
                float st[K];
#pragma unroll
                for (int r = 0; r < K; ++r) st[r] = t.stp[r];
                for (int u = tid; u < n; u += nt) {
                    float x[K];
                    ldk<K>(t.xs + (size_t)u * K, x);
                    dwt_apply<K>(x, t.thc, t.thc2, st);
                    stk<K>(t.xs + (size_t)u * K, x);
                }
                __syncthreads();
            }
        }
        if (readout_due(v, s)) tile_readout<Store, K>(v, sg.tile, t, (int)((s - 1) / v.track), true);
        if (dwt_on && ++phase == v.dwt_period) phase = 0;
    }
    seg_end<Store, K>(v, sg, t, ready);
}

template <typename Store, int K, int kMode>
__device__ __forceinline__ void run_segment(const InstView &v, const Segment &sg, unsigned char *smem,
                                            int *s_skip, int32_t *ready, int32_t *err,
                                            uint64_t wait_limit_ns)
{
    if constexpr (std::is_same<Store, uint16_t>::value)
        run_segment_q16<K, kMode>(v, sg, smem, s_skip, ready, err, wait_limit_ns);
    else
        run_segment_fp<Store, K, kMode>(v, sg, smem, s_skip, ready, err, wait_limit_ns);
}

// ---------------------------------------------------------------- sweep kernel
// One instance: CTA b runs its segment list (one whole trial per tile, or
// the head / tail pieces of the wrap-around schedule).
// Lattice tiles of up to 4 replicas, edge-list tiles of two or four replicas
// and fixed-point edge-list tiles of eight may take 1024 threads (one CTA per SM holds a large tile; more
// warps hide the dependency and record-load latency) within 64 registers;
// the others use at most 512 threads and up to 128 registers.
template <typename Store, int K, int kMode>
constexpr int max_threads()
{
    return ((kMode == MODE_LATTICE2D && K <= 4) ||
            (kMode == MODE_GENERAL && (K == 2 || K == 4) && sizeof(Store) == 4) ||
            (kMode == MODE_GENERAL && std::is_same<Store, uint16_t>::value) ||
            (kMode == MODE_GENERAL && sizeof(Store) == 2 && (K == 2 || K == 4)))
               ? 1024
               : 512;
}

template <typename Store, int K, int kMode>
__global__ void __launch_bounds__(max_threads<Store, K, kMode>()) sweep_kernel(const KernelArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_skip;
    for (int si = a.seg_off[blockIdx.x]; si < a.seg_off[blockIdx.x + 1]; ++si) {
        const Segment sg = a.segs[si];
        run_segment<Store, K, kMode>(a.v, sg, smem, &s_skip, a.ready, a.err, a.wait_limit_ns);
    }
}

// ---------------------------------------------------------------- batch kernel
// Many instances of uneven size: the instances of one (storage, K, mode)
// class share a persistent launch whose CTAs take the next unit (instance,
// tile, sweep range, flags) from a queue ordered by decreasing cost and run
// it (a whole trial, or a chunk with the state kept in global memory);
// shared memory is sized for the class's largest tile.
template <typename Store, int K, int kMode>
__global__ void __launch_bounds__(max_threads<Store, K, kMode>()) batch_kernel(const BatchArgs b)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_skip, s_unit;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(b.counter, 1);
        __syncthreads();
        const int u = s_unit;
        __syncthreads();  // all threads read s_unit before it is overwritten
        if (u >= b.n_units) break;
        const BatchUnit bu = b.units[u];
        const InstView &v = b.insts[bu.inst];
        const Segment sg{bu.tile, bu.flags, bu.s_begin, bu.s_end};
        run_segment<Store, K, kMode>(v, sg, smem, &s_skip, nullptr, nullptr, 0);
    }
}

// ---------------------------------------------------------------- finalize
// Best replica (lowest energy of its kept readout, or the largest cut when
// no energies are kept; ties -> lowest index), its energy, and its spins in
// original vertex order: the saved bits of the kept readout with tracking,
// else the rounding of the final phases at the kept bisector.
__device__ __forceinline__ uint32_t stored_q(const void *state, int storage, size_t idx)
{
    if (storage == 0) return phase_q(reinterpret_cast<const float *>(state)[idx]);
    if (storage == 1) return phase_q(__half2float(reinterpret_cast<const __half *>(state)[idx]));
    if (storage == 3) return phase_q(__bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(state)[idx]));
    return (uint32_t)reinterpret_cast<const uint16_t *>(state)[idx] << 16;
}

__device__ void finalize_body(int replicas, int K, int storage, int P, int n, int64_t W,
                              const void *state, int64_t stride, const int32_t *orig_of,
                              const int64_t *cut, const int32_t *bestp, const int64_t *energy,
                              const uint32_t *bisB, const uint32_t *bits, int words, int64_t *best,
                              int8_t *spins, int64_t target)
{
    __shared__ long long s_cut[1024];
    __shared__ int s_rep[1024];
    __shared__ unsigned long long s_hits;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) s_hits = 0;
    long long bc = LLONG_MIN;
    int br = 0x7FFFFFFF;
    unsigned long long hits = 0;
    for (int r = tid; r < replicas; r += nt) {
        const long long c = energy ? -energy[r] : cut[r];
        if (c > bc || (c == bc && r < br)) { bc = c; br = r; }
        hits += cut[r] >= target ? 1 : 0;
    }
    s_cut[tid] = bc;
    s_rep[tid] = br;
    __syncthreads();
    atomicAdd(&s_hits, hits);
    for (int o = nt / 2; o > 0; o >>= 1) {
        if (tid < o) {
            const long long c = s_cut[tid + o];
            const int r = s_rep[tid + o];
            if (c > s_cut[tid] || (c == s_cut[tid] && r < s_rep[tid])) {
                s_cut[tid] = c;
                s_rep[tid] = r;
            }
        }
        __syncthreads();
    }
    const int rb = s_rep[0];
    const long long cb = cut[rb];
    if (tid == 0) {
        best[0] = cb;
        best[1] = energy ? energy[rb] : W - 2 * cb;
        best[2] = rb;
        best[3] = (int64_t)s_hits;
    }
    if (bits) {
        const uint32_t *bw = bits + (size_t)rb * words;
        for (int v = tid; v < n; v += nt) spins[orig_of[v]] = ((bw[v >> 5] >> (v & 31)) & 1u) ? 1 : -1;
        return;
    }
    const int tile = rb / K, lane = rb % K;
    const uint32_t B = bisB ? bisB[rb] : (uint32_t)(((uint64_t)bestp[rb] << 31) / (uint64_t)P);
    for (int v = tid; v < n; v += nt) {
        const uint32_t q = stored_q(state, storage, (size_t)tile * stride + (size_t)v * K + lane);
        spins[orig_of[v]] = ((uint32_t)(q - B) < 0x80000000u) ? 1 : -1;
    }
}

__global__ void __launch_bounds__(1024) finalize_kernel(const FinalArgs a)
{
    finalize_body(a.replicas, a.K, a.storage, a.P, a.n, a.W, a.state, a.state_tile_stride, a.orig_of,
                  a.cut, a.bestp, a.energy, a.bisB, a.bits, a.words, a.best, a.spins, a.target);
}

__global__ void __launch_bounds__(1024) batch_finalize_kernel(const InstView *insts, const BatchFinal *fin)
{
    const InstView &v = insts[blockIdx.x];
    const BatchFinal &f = fin[blockIdx.x];
    finalize_body(v.replicas, v.K, f.storage, v.P, v.n, f.W, v.state, v.state_tile_stride, v.orig_of,
                  v.cut, v.bestp, v.energy, v.bisB, nullptr, 0, f.best, f.spins, LLONG_MIN);
}

// ---------------------------------------------------------------- optimal bisector
// Exact best bisector of each replica (Section II-B; the sorted sweep of
// Burer, Monteiro and Zhang 2002). With phi_v = q_v mod 2^31 and t_v the top
// bit of q_v, s_v(B) = +1 iff [B <= phi_v] xor t_v for B in [0, 2^31), so an
// edge's cut state flips on the interval (lo, hi] of its endpoints'
// positions: d_e = w_e (1 - 2 (t_i xor t_j)) enters at lo + 1 and leaves at
// hi + 1. Each vertex collects the changes that happen at its position,
// the (position, change) pairs are sorted (bitonic network over a power of
// two, in global scratch), and a block-wide prefix sum gives the cut at
// every position where it can change; the best (ties: the smallest B)
// competes with the replica's kept readout.
__global__ void __launch_bounds__(1024) opt_readout_kernel(const OptArgs o)
{
    __shared__ long long s_part[1024];
    __shared__ long long s_best[1024];
    __shared__ uint32_t s_B[1024];
    __shared__ unsigned long long s_c0;
    __shared__ int s_take;
    const InstView &v = o.v;
    const int tid = threadIdx.x, nt = blockDim.x, n = v.n, N = o.npow2;
    uint32_t *qb = o.qbuf + (size_t)blockIdx.x * n;
    int32_t *dl = o.delta + (size_t)blockIdx.x * n;
    uint64_t *it = o.items + (size_t)blockIdx.x * N;
    const int m = __ldg(v.off + v.C);
    const int storage = o.storage;
    for (int r = blockIdx.x; r < v.replicas; r += gridDim.x) {
        const int tile = r / v.K, lane = r % v.K;
        if (tid == 0) s_c0 = 0ull;
        for (int u = tid; u < n; u += nt) {
            qb[u] = stored_q(v.state, storage, (size_t)tile * v.state_tile_stride + (size_t)u * v.K + lane);
            dl[u] = 0;
        }
        __syncthreads();
        long long c0 = 0;
        for (int e = tid; e < m; e += nt) {
            const uint32_t rec = load_rec(v, e);
            const int wv = (int)__ldg(v.w + e);
            const int i = (int)(rec & 0xFFFFu), j = (int)(rec >> 16);
            const uint32_t qi = qb[i], qj = qb[j];
            const bool cross = ((qi ^ qj) >> 31) != 0;
            if (cross) c0 += wv;
            const uint32_t pi = qi & 0x7FFFFFFFu, pj = qj & 0x7FFFFFFFu;
            if (pi == pj) continue;
            const int d = cross ? -wv : wv;
            atomicAdd(dl + (pi < pj ? i : j), d);
            atomicAdd(dl + (pi < pj ? j : i), -d);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) c0 += __shfl_xor_sync(0xFFFFFFFFu, c0, off);
        if ((tid & 31) == 0) atomicAdd(&s_c0, (unsigned long long)c0);
        __syncthreads();
        for (int u = tid; u < N; u += nt)
            it[u] = u < n ? ((uint64_t)(qb[u] & 0x7FFFFFFFu) << 32) | (uint32_t)dl[u] : 0xFFFFFFFF00000000ull;
        __syncthreads();
        for (int k = 2; k <= N; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < N; i += nt) {
                    const int l = i ^ j;
                    if (l > i) {
                        const uint64_t x = it[i], y = it[l];
                        if ((x > y) == ((i & k) == 0)) {
                            it[i] = y;
                            it[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // block prefix sum over contiguous chunks of the sorted pairs
        const int chunk = (n + nt - 1) / nt;
        const int a0 = min(n, tid * chunk), a1 = min(n, a0 + chunk);
        long long sum = 0;
        for (int i = a0; i < a1; ++i) sum += (int32_t)(uint32_t)it[i];
        s_part[tid] = sum;
        __syncthreads();
        if (tid == 0) {
            long long acc = 0;
            for (int i = 0; i < nt; ++i) {
                const long long t0 = s_part[i];
                s_part[i] = acc;
                acc += t0;
            }
        }
        __syncthreads();
        const long long C0 = (long long)s_c0;
        long long run = C0 + s_part[tid], best = LLONG_MIN;
        uint32_t bB = 0xFFFFFFFFu;
        if (tid == 0) { best = C0; bB = 0; }
        for (int i = a0; i < a1; ++i) {
            const uint64_t x = it[i];
            run += (int32_t)(uint32_t)x;
            const uint32_t pos = (uint32_t)(x >> 32);
            const bool end = (i == n - 1) || ((uint32_t)(it[i + 1] >> 32) != pos);
            if (end && pos + 1u < 0x80000000u && run > best) {
                best = run;
                bB = pos + 1u;
            }
        }
        s_best[tid] = best;
        s_B[tid] = bB;
        __syncthreads();
        for (int off = nt / 2; off > 0; off >>= 1) {
            if (tid < off) {
                const long long c = s_best[tid + off];
                const uint32_t b2 = s_B[tid + off];
                if (c > s_best[tid] || (c == s_best[tid] && b2 < s_B[tid])) {
                    s_best[tid] = c;
                    s_B[tid] = b2;
                }
            }
            __syncthreads();
        }
        const long long cut = s_best[0];
        const uint32_t B = s_B[0];
        if (tid == 0) {
            const long long E = v.W - 2 * cut;
            const int take = !o.keep_better || !v.energy || E < v.energy[r];
            if (take) {
                v.cut[r] = cut;
                v.bestp[r] = -1;
                if (v.energy) v.energy[r] = E;
                if (v.bisB) v.bisB[r] = B;
            }
            s_take = take;
        }
        __syncthreads();
        if (s_take && v.bits) {
            for (int wi = tid; wi < v.words; wi += nt) {
                uint32_t word = 0u;
                const int v0 = wi * 32, v1 = min(n, v0 + 32);
                for (int u = v0; u < v1; ++u)
                    if ((uint32_t)(qb[u] - B) < 0x80000000u) word |= 1u << (u - v0);
                v.bits[(size_t)r * v.words + wi] = word;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side
template <typename Store, int K, int M>
static int launch_one(const LaunchCfg &cfg, const KernelArgs &a, void *stream)
{
    auto fn = sweep_kernel<Store, K, M>;
    static size_t set_bytes = 0;
    if (cfg.smem > 48 * 1024 && cfg.smem > set_bytes) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem) !=
            cudaSuccess)
            return -1;
        set_bytes = cfg.smem;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cfg.cooperative) {
        void *args[] = {const_cast<KernelArgs *>(&a)};
        return cudaLaunchCooperativeKernel((const void *)fn, dim3(cfg.grid), dim3(cfg.threads), args,
                                           cfg.smem, st) == cudaSuccess ? 0 : -1;
    }
    fn<<<cfg.grid, cfg.threads, cfg.smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename Store, int K, int M>
static int occ_one(int threads, size_t smem)
{
    auto fn = sweep_kernel<Store, K, M>;
    if (threads < 1 || threads > max_threads<Store, K, M>()) return 0;  // beyond the launch bound
    if (smem > 48 * 1024)
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            cudaGetLastError();  // leave no error behind for the next launch check
            return 0;
        }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

#define COSM_DISPATCH_M(T, KK, MODE, CALL)                 \
    do {                                                   \
        if ((MODE) == MODE_GENERAL) return CALL(T, KK, 0); \
        if ((MODE) == MODE_ACCUM) return CALL(T, KK, 1);   \
        if ((MODE) == MODE_LATTICE2D) return CALL(T, KK, 2); \
    } while (0)

#define COSM_DISPATCH(STORAGE, K, MODE, CALL)                       \
    do {                                                            \
        if ((STORAGE) == 0) {                                       \
            if ((K) == 1) COSM_DISPATCH_M(float, 1, MODE, CALL);    \
            if ((K) == 2) COSM_DISPATCH_M(float, 2, MODE, CALL);    \
            if ((K) == 4) COSM_DISPATCH_M(float, 4, MODE, CALL);    \
        } else if ((STORAGE) == 1) {                                \
            if ((K) == 2) COSM_DISPATCH_M(__half, 2, MODE, CALL);   \
            if ((K) == 4) COSM_DISPATCH_M(__half, 4, MODE, CALL);   \
            if ((K) == 8) COSM_DISPATCH_M(__half, 8, MODE, CALL);   \
        } else if ((STORAGE) == 3) {                                \
            if ((K) == 2) COSM_DISPATCH_M(__nv_bfloat16, 2, MODE, CALL); \
            if ((K) == 4) COSM_DISPATCH_M(__nv_bfloat16, 4, MODE, CALL); \
            if ((K) == 8) COSM_DISPATCH_M(__nv_bfloat16, 8, MODE, CALL); \
        } else {                                                    \
            if ((K) == 2) COSM_DISPATCH_M(uint16_t, 2, MODE, CALL); \
            if ((K) == 4) COSM_DISPATCH_M(uint16_t, 4, MODE, CALL); \
            if ((K) == 8) COSM_DISPATCH_M(uint16_t, 8, MODE, CALL); \
        }                                                           \
    } while (0)

size_t sweep_smem_bytes(int storage, int K, int n, int P, int mode)
{
#define SMEM_CALL(T, KK, M) smem_bytes<T, KK>(n, P, (M) == MODE_ACCUM)
    COSM_DISPATCH(storage, K, mode, SMEM_CALL);
#undef SMEM_CALL
    return 0;
}

int sweep_occupancy(int storage, int K, int mode, int threads, size_t smem)
{
#define OCC_CALL(T, KK, M) occ_one<T, KK, M>(threads, smem)
    COSM_DISPATCH(storage, K, mode, OCC_CALL);
#undef OCC_CALL
    return 0;
}

int sweep_launch(const LaunchCfg &cfg, const KernelArgs &a, void *stream)
{
#define LAUNCH_CALL(T, KK, M) launch_one<T, KK, M>(cfg, a, stream)
    COSM_DISPATCH(cfg.storage, cfg.K, cfg.mode, LAUNCH_CALL);
#undef LAUNCH_CALL
    return -1;
}

int finalize_launch(const FinalArgs &a, void *stream)
{
    finalize_kernel<<<1, 1024, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int opt_readout_launch(const OptArgs &a, int grid, void *stream)
{
    opt_readout_kernel<<<grid, 1024, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Raises a batch kernel's dynamic shared-memory limit once per size (not
// again while a launch is being captured into a graph).
template <typename Store, int K, int M>
static int batch_set_smem(size_t smem)
{
    static size_t set_bytes = 0;
    if (smem > 48 * 1024 && smem > set_bytes) {
        if (cudaFuncSetAttribute(batch_kernel<Store, K, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess) {
            cudaGetLastError();  // leave no error behind for the next launch check
            return -1;
        }
        set_bytes = smem;
    }
    return 0;
}

template <typename Store, int K, int M>
static int batch_occ_one(int threads, size_t smem)
{
    auto fn = batch_kernel<Store, K, M>;
    if (threads < 1 || threads > max_threads<Store, K, M>()) return 0;  // beyond the launch bound
    if (batch_set_smem<Store, K, M>(smem)) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

template <typename Store, int K, int M>
static int batch_launch_one(int grid, int threads, size_t smem, const BatchArgs &b, void *stream)
{
    auto fn = batch_kernel<Store, K, M>;
    if (batch_set_smem<Store, K, M>(smem)) return -1;
    fn<<<grid, threads, smem, reinterpret_cast<cudaStream_t>(stream)>>>(b);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int batch_occupancy(int storage, int K, int mode, int threads, size_t smem)
{
#define BOCC_CALL(T, KK, M) batch_occ_one<T, KK, M>(threads, smem)
    COSM_DISPATCH(storage, K, mode, BOCC_CALL);
#undef BOCC_CALL
    return 0;
}

int batch_launch(int storage, int K, int mode, int grid, int threads, size_t smem, const BatchArgs &b,
                 void *stream)
{
#define BLAUNCH_CALL(T, KK, M) batch_launch_one<T, KK, M>(grid, threads, smem, b, stream)
    COSM_DISPATCH(storage, K, mode, BLAUNCH_CALL);
#undef BLAUNCH_CALL
    return -1;
}

int batch_finalize_launch(int count, const InstView *insts, const BatchFinal *fin, void *stream)
{
    batch_finalize_kernel<<<count, 1024, 0, reinterpret_cast<cudaStream_t>(stream)>>>(insts, fin);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace cosm


// ---------------------------------------------------------------- SMEM probe
namespace cosm {

// Shared-memory read bandwidth: every thread streams 16-byte words from a
// conflict-free pattern; thread 0 records the SM clocks spent.
__global__ void __launch_bounds__(1024) smem_probe_kernel(int iters, unsigned long long *clk,
                                                          uint32_t *sink)
{
    __shared__ uint4 buf[4096];
    const int tid = threadIdx.x;
    for (int k = tid; k < 4096; k += blockDim.x) buf[k] = make_uint4(k, k + 1, k + 2, k + 3);
    __syncthreads();
    unsigned long long t0 = clock64();
    uint32_t acc = 0;
    int idx = tid;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint4 v = buf[(idx + u * 512) & 4095];
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
        idx += 7;
    }
    __syncthreads();
    unsigned long long t1 = clock64();
    if (tid == 0) atomicMax(clk, t1 - t0);
    if (acc == 0xFFFFFFFFu) sink[0] = acc;
}

}  // namespace cosm

extern "C" int cosm_probe_smem(int32_t iters, double *bytes_per_clk_per_sm, double *gbps)
{
    using namespace cosm;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return COSM_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned long long *clk = nullptr;
    uint32_t *sink = nullptr;
    if (cudaMalloc(&clk, 8) != cudaSuccess || cudaMalloc(&sink, 4) != cudaSuccess) return COSM_ERR_NOMEM;
    cudaMemset(clk, 0, 8);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 1024, blocks = 2 * sms;
    smem_probe_kernel<<<blocks, threads>>>(iters / 4 + 1, clk, sink);  // warm-up
    cudaMemset(clk, 0, 8);
    cudaEventRecord(e0);
    smem_probe_kernel<<<blocks, threads>>>(iters, clk, sink);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long cycles = 0;
    cudaMemcpy(&cycles, clk, 8, cudaMemcpyDeviceToHost);
    cudaFree(clk);
    cudaFree(sink);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return COSM_ERR_CUDA;
    const double bytes_per_cta = (double)threads * iters * 8 * 16;
    // two CTAs share an SM; clk is the longest CTA's span
    if (bytes_per_clk_per_sm) *bytes_per_clk_per_sm = 2.0 * bytes_per_cta / (double)cycles;
    if (gbps) *gbps = bytes_per_cta * blocks / (ms * 1e-3) / 1e9;
    return COSM_OK;
}

// ---------------------------------------------------------------- FP32 issue probe
namespace cosm {

// FP32 arithmetic issue rate: every thread runs 8 independent chains of
// fused multiply-adds, scalar (fma.rn.f32, one operation per lane) or packed
// (fma.rn.f32x2, two operations per lane); thread 0 records the SM clocks
// spent. The chains hold values near a fixed point of x -> a x + b, so no
// lane overflows or goes subnormal.
template <bool kPacked>
__global__ void __launch_bounds__(1024) fp32_probe_kernel(int iters, unsigned long long *clk, float *sink)
{
    const float a = 0.5f, b = 0.25f + 1e-3f * (float)(threadIdx.x & 7);
    f32x2 x2[8];
    float x1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        x1[i] = 0.125f * (float)i;
        x2[i] = p_pack(x1[i], -x1[i]);
    }
    const f32x2 a2 = p_pack(a, a), b2 = p_pack(b, b);
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if constexpr (kPacked) {
                    x2[i] = p_fma(x2[i], a2, b2);
                } else {
                    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x1[i]) : "f"(a), "f"(b));
                }
            }
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    if (threadIdx.x == 0) atomicMax(clk, t1 - t0);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += kPacked ? p_lo(x2[i]) + p_hi(x2[i]) : x1[i];
    if (s == 12345.0f) sink[0] = s;
}

}  // namespace cosm

extern "C" int cosm_probe_fp32(int32_t iters, double *ops_per_clk_per_sm, double *ops_per_clk_per_sm_packed)
{
    using namespace cosm;
    if (iters < 1) return COSM_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return COSM_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned long long *clk = nullptr;
    float *sink = nullptr;
    if (cudaMalloc(&clk, 8) != cudaSuccess) return COSM_ERR_NOMEM;
    if (cudaMalloc(&sink, 4) != cudaSuccess) {
        cudaFree(clk);
        return COSM_ERR_NOMEM;
    }
    const int threads = 1024, blocks = 2 * sms;
    // operations per CTA: threads x iters x 8 unrolled x 8 chains (x 2 packed)
    const double ops = (double)threads * iters * 64.0;
    double res[2] = {0.0, 0.0};
    cudaError_t err = cudaSuccess;
    for (int packed = 0; packed < 2 && err == cudaSuccess; ++packed) {
        for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
            cudaMemset(clk, 0, 8);
            if (packed) fp32_probe_kernel<true><<<blocks, threads>>>(rep ? iters : iters / 4 + 1, clk, sink);
            else fp32_probe_kernel<false><<<blocks, threads>>>(rep ? iters : iters / 4 + 1, clk, sink);
        }
        err = cudaDeviceSynchronize();
        unsigned long long cycles = 0;
        if (err == cudaSuccess) err = cudaMemcpy(&cycles, clk, 8, cudaMemcpyDeviceToHost);
        // two CTAs share an SM; clk is the longest CTA's span
        if (cycles) res[packed] = 2.0 * ops * (packed ? 2.0 : 1.0) / (double)cycles;
    }
    cudaFree(clk);
    cudaFree(sink);
    if (err != cudaSuccess) return COSM_ERR_CUDA;
    if (ops_per_clk_per_sm) *ops_per_clk_per_sm = res[0];
    if (ops_per_clk_per_sm_packed) *ops_per_clk_per_sm_packed = res[1];
    return COSM_OK;
}
