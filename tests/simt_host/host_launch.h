// Test harness only: kernel launches on host threads (one std::thread per
// CUDA thread, all blocks of a launch at once, shared memory per block filled
// with garbage first) and raw file output, for the drivers of this directory.
#pragma once
#include <memory>
#include <string>
#include <thread>
#include "cuda_runtime.h"

thread_local uint3 threadIdx, blockIdx;
dim3 blockDim, gridDim;
namespace emu {
Block* blocks = nullptr;
Warp* warps = nullptr;
unsigned char* smem_base = nullptr;
size_t smem_per_block = 0;
thread_local std::vector<Pending> pending;
std::atomic<unsigned long long> site_warnings{0};
}  // namespace emu

template <class F>
static void launch(unsigned nblocks, unsigned threads, size_t smem, F body)
{
    gridDim = dim3{nblocks, 1, 1};
    blockDim = dim3{threads, 1, 1};
    std::unique_ptr<emu::Block[]> b(new emu::Block[nblocks]);
    std::unique_ptr<emu::Warp[]> w(new emu::Warp[(size_t)nblocks * 32]);
    std::vector<unsigned char> sm((size_t)nblocks * smem + 64);
    std::memset(sm.data(), 0xA5, sm.size());   // shared memory starts undefined
    emu::blocks = b.get();
    emu::warps = w.get();
    emu::smem_base = reinterpret_cast<unsigned char*>(((uintptr_t)sm.data() + 15) & ~(uintptr_t)15);
    emu::smem_per_block = smem;
    std::vector<std::thread> th;
    for (unsigned bi = 0; bi < nblocks; ++bi)
        for (unsigned t = 0; t < threads; ++t)
            th.emplace_back([=] {
                threadIdx = uint3{t, 0, 0};
                blockIdx = uint3{bi, 0, 0};
                body();
                emu::bulk_wait();
                emu::thread_exit();
            });
    for (auto& x : th) x.join();
}

template <class T> static void dump(const std::string& path, const T* p, size_t n)
{
    FILE* f = std::fopen(path.c_str(), "wb");
    std::fwrite(p, sizeof(T), n, f);
    std::fclose(f);
}

template <class T> static std::vector<T> load(const std::string& path)
{
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) { std::fprintf(stderr, "cannot open %s\n", path.c_str()); std::exit(2); }
    std::fseek(f, 0, SEEK_END);
    const long n = std::ftell(f);
    std::fseek(f, 0, SEEK_SET);
    std::vector<T> v((size_t)n / sizeof(T));
    if (std::fread(v.data(), 1, (size_t)n, f) != (size_t)n) std::exit(2);
    std::fclose(f);
    return v;
}
