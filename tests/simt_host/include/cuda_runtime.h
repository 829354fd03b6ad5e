// Test harness only: a host stand-in for the CUDA device features the
// engine's kernels use, so that their source can be compiled with g++ and
// run on host threads under ThreadSanitizer, AddressSanitizer and
// UndefinedBehaviorSanitizer (compute-sanitizer is not available to this
// project).  Every lane is a std::thread; a warp collective (__syncwarp,
// __ballot_sync, __shfl*_sync, __reduce_add_sync) is a rendezvous of the
// lanes named in its mask under one mutex per warp, which gives the
// sanitizers the same ordering the hardware collective gives; a lane outside
// the mask, a source lane outside the mask, lanes of one mask that meet at
// different kinds of collective (a ballot and a shuffle, say) or a
// collective that never completes aborts the run, and lanes that meet at the
// same kind of collective from different source lines are reported on
// stderr ("EMU WARNING") and counted.  Shared-memory atomics are host atomics.  A bulk
// asynchronous copy (cp.async.bulk) is performed at its wait, the latest
// moment the hardware may read its source, so a source rewritten too early
// shows up as wrong output.  The product library never includes this file.
#pragma once
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <cassert>
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <atomic>
#include <condition_variable>
#include <thread>
#include <chrono>
#include <vector>
#define __device__
#define __global__
#define __host__
#define __shared__
#define __constant__
#define __forceinline__ inline __attribute__((always_inline))
#define __noinline__ __attribute__((noinline))
#define __align__(n) __attribute__((aligned(n)))
#define __launch_bounds__(...)
#define __restrict__ __restrict
struct uint3 { unsigned x, y, z; };
struct dim3 { unsigned x, y, z; };
extern thread_local uint3 threadIdx, blockIdx;
extern dim3 blockDim, gridDim;
struct uint4 { unsigned x, y, z, w; };
struct uint2 { unsigned x, y; };
struct int4 { int x, y, z, w; };
struct int2 { int x, y; };
inline uint4 make_uint4(unsigned a, unsigned b, unsigned c, unsigned d) { return uint4{a, b, c, d}; }
inline uint2 make_uint2(unsigned a, unsigned b) { return uint2{a, b}; }
inline int4 make_int4(int a, int b, int c, int d) { return int4{a, b, c, d}; }
inline int2 make_int2(int a, int b) { return int2{a, b}; }
using std::min;
using std::max;
typedef struct CUstream_st* cudaStream_t;
typedef struct CUgraphExec_st* cudaGraphExec_t;
typedef int cudaError_t;

namespace emu {
// The kind of a warp collective: lanes of one mask that meet must all be at
// the same kind (on the hardware, lanes of one mask at different collectives
// is undefined behaviour and can hang or corrupt values).
enum Op : int { kOpSync = 1, kOpBallot, kOpReduce, kOpShfl, kOpShflUp, kOpShflDown, kOpShflXor };
inline const char* op_name(int op)
{
    static const char* names[] = {"?", "syncwarp", "ballot", "reduce", "shfl", "shfl_up", "shfl_down", "shfl_xor"};
    return names[op >= 0 && op < 8 ? op : 0];
}
struct Rendezvous {
    unsigned arrived = 0;
    int phase = 0;            // 0 collecting, 1 reading
    int readers = 0;
    unsigned long long gen = 0;
    unsigned long long vals[32];
    int op = 0;               // the collective of the first lane to arrive in this round
    const char* file = nullptr;
    int line = 0;
};
extern std::atomic<unsigned long long> site_warnings;
struct Warp {
    std::mutex m;
    std::condition_variable cv;
    std::map<unsigned, Rendezvous> rv;
};
struct Block {                    // __syncthreads: every thread of the block that has not returned
    std::mutex m;
    std::condition_variable cv;
    unsigned arrived = 0, exited = 0;
    unsigned long long gen = 0;
    std::map<int, void*> statics;  // the block's static __shared__ variables, by source line
    ~Block() { for (auto& kv : statics) std::free(kv.second); }
};
extern Block* blocks;             // [blocks], allocated per launch
extern Warp* warps;              // [blocks][32 warps], allocated per launch
extern unsigned char* smem_base;  // [blocks][smem_per_block]
extern size_t smem_per_block;
inline Warp& warp_of() { return warps[blockIdx.x * 32 + (threadIdx.x >> 5)]; }
inline unsigned char* block_smem() { return smem_base + (size_t)blockIdx.x * smem_per_block; }
[[noreturn]] inline void fail(const char* what, unsigned mask)
{
    std::fprintf(stderr, "EMU FAILURE: %s (lane %u, mask %08x)\n", what, threadIdx.x & 31, mask);
    std::fflush(stderr);
    std::abort();
}
template <class F>
unsigned long long exchange(unsigned mask, unsigned long long v, F f, int op, const char* file, int line)
{
    const unsigned lane = threadIdx.x & 31;
    if (!((mask >> lane) & 1u)) fail("calling lane not in mask", mask);
    Warp& W = warp_of();
    std::unique_lock<std::mutex> lk(W.m);
    Rendezvous& R = W.rv[mask];
    W.cv.wait(lk, [&] { return R.phase == 0; });
    if ((R.arrived >> lane) & 1u) fail("lane arrived twice", mask);
    if (R.arrived == 0) {
        R.op = op; R.file = file; R.line = line;
    } else if (R.op != op) {
        std::fprintf(stderr, "EMU FAILURE: lanes of one mask met at different collectives: %s at %s:%d and %s at %s:%d\n",
                     op_name(R.op), R.file, R.line, op_name(op), file, line);
        fail("mismatched collectives", mask);
    } else if (R.line != line || std::strcmp(R.file, file) != 0) {
        std::fprintf(stderr, "EMU WARNING: lanes of one mask met at one collective (%s) from different sites: %s:%d and %s:%d\n",
                     op_name(op), R.file, R.line, file, line);
        site_warnings++;
    }
    R.vals[lane] = v;
    R.arrived |= 1u << lane;
    const unsigned long long my = R.gen;
    if (R.arrived == mask) {
        R.phase = 1;
        R.readers = __builtin_popcount(mask);
        W.cv.notify_all();
    } else {
        if (!W.cv.wait_for(lk, std::chrono::seconds(20), [&] { return R.phase == 1 && R.gen == my; }))
            fail("collective never completed (deadlock)", mask);
    }
    const unsigned long long out = f(R.vals, lane);
    if (--R.readers == 0) {
        R.arrived = 0;
        R.phase = 0;
        R.gen++;
        W.cv.notify_all();
    }
    return out;
}
inline unsigned src_ok(unsigned mask, unsigned s)
{
    if (!((mask >> s) & 1u)) fail("source lane not in mask", mask);
    return s;
}
template <class T> unsigned long long bits(T v) { unsigned long long u = 0; std::memcpy(&u, &v, sizeof(T)); return u; }
template <class T> T from(unsigned long long u) { T v; std::memcpy(&v, &u, sizeof(T)); return v; }
// bulk copies: performed at the wait (the latest moment the hardware may read)
struct Pending { void* dst; const void* src; size_t n; };
extern thread_local std::vector<Pending> pending;
inline void bulk_copy(void* dst, const void* src, size_t n) { pending.push_back({dst, src, n}); }
inline void bulk_wait() { for (auto& p : pending) std::memcpy(p.dst, p.src, p.n); pending.clear(); }
}  // namespace emu

#define EMU_SITE const char* file_ = __builtin_FILE(), int line_ = __builtin_LINE()
inline void __syncwarp(unsigned mask = 0xffffffffu, EMU_SITE)
{
    emu::exchange(mask, 0, [](auto*, unsigned) { return 0ull; }, emu::kOpSync, file_, line_);
}
inline unsigned __ballot_sync(unsigned mask, int p, EMU_SITE)
{
    return (unsigned)emu::exchange(mask, p != 0, [mask](unsigned long long* v, unsigned) {
        unsigned long long b = 0;
        for (int l = 0; l < 32; ++l) if (((mask >> l) & 1u) && v[l]) b |= 1ull << l;
        return b; }, emu::kOpBallot, file_, line_);
}
inline int __any_sync(unsigned mask, int p, EMU_SITE) { return __ballot_sync(mask, p, file_, line_) != 0; }
inline int __all_sync(unsigned mask, int p, EMU_SITE) { return __ballot_sync(mask, p, file_, line_) == mask; }
inline unsigned __reduce_add_sync(unsigned mask, unsigned v, EMU_SITE)
{
    return (unsigned)emu::exchange(mask, v, [mask](unsigned long long* x, unsigned) {
        unsigned s = 0;
        for (int l = 0; l < 32; ++l) if ((mask >> l) & 1u) s += (unsigned)x[l];
        return (unsigned long long)s; }, emu::kOpReduce, file_, line_);
}
template <class T> T __shfl_sync(unsigned mask, T v, int src, int width = 32, EMU_SITE)
{
    return emu::from<T>(emu::exchange(mask, emu::bits(v), [mask, src, width](unsigned long long* x, unsigned lane) {
        const unsigned s = (lane & ~(unsigned)(width - 1)) | ((unsigned)src & (unsigned)(width - 1));
        return x[emu::src_ok(mask, s)]; }, emu::kOpShfl, file_, line_));
}
template <class T> T __shfl_up_sync(unsigned mask, T v, unsigned d, int width = 32, EMU_SITE)
{
    return emu::from<T>(emu::exchange(mask, emu::bits(v), [mask, d, width](unsigned long long* x, unsigned lane) {
        const unsigned s = (lane & (unsigned)(width - 1)) >= d ? lane - d : lane;
        return x[emu::src_ok(mask, s)]; }, emu::kOpShflUp, file_, line_));
}
template <class T> T __shfl_down_sync(unsigned mask, T v, unsigned d, int width = 32, EMU_SITE)
{
    return emu::from<T>(emu::exchange(mask, emu::bits(v), [mask, d, width](unsigned long long* x, unsigned lane) {
        const unsigned s = (lane & (unsigned)(width - 1)) + d < (unsigned)width ? lane + d : lane;
        return x[emu::src_ok(mask, s)]; }, emu::kOpShflDown, file_, line_));
}
template <class T> T __shfl_xor_sync(unsigned mask, T v, int m, int width = 32, EMU_SITE)
{
    return emu::from<T>(emu::exchange(mask, emu::bits(v), [mask, m, width](unsigned long long* x, unsigned lane) {
        unsigned s = lane ^ (unsigned)m;
        if ((s & ~(unsigned)(width - 1)) > (lane & ~(unsigned)(width - 1))) s = lane;
        return x[emu::src_ok(mask, s)]; }, emu::kOpShflXor, file_, line_));
}
inline int __popc(unsigned v) { return __builtin_popcount(v); }
inline int __popcll(unsigned long long v) { return __builtin_popcountll(v); }
inline int __ffs(int v) { return __builtin_ffs(v); }
inline int __ffsll(long long v) { return __builtin_ffsll(v); }
inline int __clz(int v) { return v == 0 ? 32 : __builtin_clz((unsigned)v); }
inline int __clzll(long long v) { return v == 0 ? 64 : __builtin_clzll((unsigned long long)v); }
inline unsigned __umulhi(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }
// dot product of the four bytes of a and b, plus c
inline unsigned __dp4a(unsigned a, unsigned b, unsigned c)
{
    for (int i = 0; i < 4; ++i) c += ((a >> (8 * i)) & 0xFFu) * ((b >> (8 * i)) & 0xFFu);
    return c;
}
// per byte: 0xFF where the byte of a is above the byte of b (unsigned), else 0
inline unsigned __vcmpgtu4(unsigned a, unsigned b)
{
    unsigned r = 0;
    for (int i = 0; i < 4; ++i)
        if (((a >> (8 * i)) & 0xFFu) > ((b >> (8 * i)) & 0xFFu)) r |= 0xFFu << (8 * i);
    return r;
}
inline unsigned __brev(unsigned v) { unsigned r = 0; for (int i = 0; i < 32; ++i) r |= ((v >> i) & 1u) << (31 - i); return r; }
template <class T> T atomicOr(T* p, T v) { return __atomic_fetch_or(p, v, __ATOMIC_SEQ_CST); }
template <class T> T atomicAnd(T* p, T v) { return __atomic_fetch_and(p, v, __ATOMIC_SEQ_CST); }
template <class T> T atomicAdd(T* p, T v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
template <class T> T atomicSub(T* p, T v) { return __atomic_fetch_sub(p, v, __ATOMIC_SEQ_CST); }
template <class T> T atomicExch(T* p, T v) { return __atomic_exchange_n(p, v, __ATOMIC_SEQ_CST); }
template <class T> T atomicCAS(T* p, T c, T v) { __atomic_compare_exchange_n(p, &c, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST); return c; }
template <class T> T atomicMin(T* p, T v) { T o = __atomic_load_n(p, __ATOMIC_SEQ_CST); while (v < o && !__atomic_compare_exchange_n(p, &o, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) {} return o; }
template <class T> T atomicMax(T* p, T v) { T o = __atomic_load_n(p, __ATOMIC_SEQ_CST); while (v > o && !__atomic_compare_exchange_n(p, &o, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) {} return o; }
namespace emu {
// A static __shared__ variable: one object per block (first use allocates it,
// filled with garbage like uninitialised shared memory).
template <class T> T* block_static(int key)
{
    Block& B = blocks[blockIdx.x];
    std::lock_guard<std::mutex> lk(B.m);
    auto it = B.statics.find(key);
    if (it == B.statics.end()) {
        void* p = std::aligned_alloc(64, (sizeof(T) + 63) / 64 * 64);
        std::memset(p, 0xA5, sizeof(T));
        it = B.statics.emplace(key, p).first;
    }
    return reinterpret_cast<T*>(it->second);
}
}  // namespace emu
inline void __syncthreads()
{
    emu::Block& B = emu::blocks[blockIdx.x];
    std::unique_lock<std::mutex> lk(B.m);
    const unsigned long long my = B.gen;
    if (++B.arrived + B.exited == blockDim.x) {
        B.arrived = 0;
        B.gen++;
        B.cv.notify_all();
    } else if (!B.cv.wait_for(lk, std::chrono::seconds(20), [&] { return B.gen != my; })) {
        emu::fail("__syncthreads never completed", 0);
    }
}
namespace emu {
inline void thread_exit()         // a returned thread no longer holds up __syncthreads
{
    Block& B = blocks[blockIdx.x];
    std::lock_guard<std::mutex> lk(B.m);
    ++B.exited;
    if (B.arrived > 0 && B.arrived + B.exited == blockDim.x) {
        B.arrived = 0;
        B.gen++;
        B.cv.notify_all();
    }
}
}  // namespace emu
inline float __fdiv_rn(float a, float b) { return a / b; }
inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
inline double __dadd_rn(double a, double b) { return a + b; }
inline double __dmul_rn(double a, double b) { return a * b; }
inline double __ddiv_rn(double a, double b) { return a / b; }
inline double __longlong_as_double(long long v) { double d; std::memcpy(&d, &v, 8); return d; }
inline long long __double_as_longlong(double d) { long long v; std::memcpy(&v, &d, 8); return v; }
// runtime calls reached by host helpers next to the kernels
enum { cudaSuccess = 0 };
inline cudaError_t cudaGetDevice(int* d) { *d = 0; return 0; }
inline cudaError_t cudaGetLastError() { return 0; }
template <class K> inline cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessor(int* n, K, int, size_t) { *n = 1; return 0; }
inline void __threadfence() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
inline void __threadfence_system() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
// a real sleep: a bounded wait keeps its bound in time however slowly the
// host threads run (at least the timer's granularity per call)
inline void __nanosleep(unsigned ns) { std::this_thread::sleep_for(std::chrono::nanoseconds(ns)); }
inline unsigned long long __cvta_generic_to_shared(const void* p) { return (unsigned long long)(uintptr_t)p; }
