// Test harness only: runs the env's reset kernel and its persistent step
// kernel (k_env_run) on host threads through include/cuda_runtime.h of this
// directory.  N slots, S plies in one launch of `blocks` blocks of `wpb`
// warps with teams of L lanes, every ply's outputs kept (ring of S rows) and
// written to <out>.{action,reward,done,ply,mask,stats} for comparison with
// the oracle.
//   env_on_host N S L wpb gpf blocks seed out
#include <thread>
#include <memory>
#include <string>
#include "cuda_runtime.h"
thread_local uint3 threadIdx, blockIdx;
dim3 blockDim, gridDim;
namespace emu {
Warp* warps = nullptr;
unsigned char* smem_base = nullptr;
size_t smem_per_block = 0;
thread_local std::vector<Pending> pending;
}
#include "env_dev.cu"

template <class F>
static void launch(unsigned blocks, unsigned threads, size_t smem, F body)
{
    gridDim = dim3{blocks, 1, 1};
    blockDim = dim3{threads, 1, 1};
    std::unique_ptr<emu::Warp[]> w(new emu::Warp[(size_t)blocks * 32]);
    std::vector<unsigned char> sm((size_t)blocks * smem + 64);
    std::memset(sm.data(), 0xA5, sm.size());   // uninitialised shared memory
    emu::warps = w.get();
    emu::smem_base = reinterpret_cast<unsigned char*>(((uintptr_t)sm.data() + 15) & ~(uintptr_t)15);
    emu::smem_per_block = smem;
    std::vector<std::thread> th;
    for (unsigned b = 0; b < blocks; ++b)
        for (unsigned t = 0; t < threads; ++t)
            th.emplace_back([=] { threadIdx = uint3{t, 0, 0}; blockIdx = uint3{b, 0, 0}; body(); emu::bulk_wait(); });
    for (auto& x : th) x.join();
}

template <class T> static void dump(const std::string& path, const T* p, size_t n)
{
    FILE* f = std::fopen(path.c_str(), "wb");
    std::fwrite(p, sizeof(T), n, f);
    std::fclose(f);
}

template <int L>
static void run(EnvArgs a, int32_t* queue, int S, int gpf, int wpb, int blocks, int16_t* act, int8_t* rew, uint8_t* done,
                int16_t* ply, uint8_t* mask)
{
    const size_t sm = (size_t)wpb * (32 / L) * sizeof(SmemGame);
    launch(blocks, 32 * wpb, sm, [=] { k_env_run<L, false>(a, queue, S, S, gpf, act, rew, done, ply, mask); });
}

int main(int argc, char** argv)
{
    const int N = std::atoi(argv[1]), S = std::atoi(argv[2]), L = std::atoi(argv[3]), wpb = std::atoi(argv[4]);
    const int gpf = std::atoi(argv[5]), blocks = std::atoi(argv[6]);
    const unsigned long long seed = std::strtoull(argv[7], nullptr, 10);
    const std::string out = argv[8];
    std::vector<GameCore> core(N);
    std::vector<uint16_t> ring((size_t)N * kRing);
    std::vector<uint64_t> pi((size_t)N * kPiWords);
    std::vector<uint32_t> stats((size_t)N * 8);
    int32_t status[2] = {0, 0x7FFFFFFF};
    int32_t queue = 0;
    EnvArgs a{};
    a.core = core.data(); a.ring = ring.data(); a.pi = pi.data(); a.stats = stats.data(); a.status = status;
    a.N = N; a.k0 = (uint32_t)seed; a.k1 = (uint32_t)(seed >> 32);
    a.R.k = 100; a.R.cap = 1000; a.R.flags = kTwoSquare | kChase | kAutoreset;
    a.reset = ResetSrc{nullptr, nullptr, nullptr, 0, 0};
    a.hist = nullptr; a.now = nullptr; a.H = 0;
    // creation: every slot reset (teams of 32, 4 per block)
    launch((N + 3) / 4, 128, 4 * sizeof(SmemGame), [=] { k_env_reset(a, nullptr, nullptr, 1); });
    std::vector<int16_t> act((size_t)S * N), ply((size_t)S * N);
    std::vector<int8_t> rew((size_t)S * N);
    std::vector<uint8_t> done((size_t)S * N), mask((size_t)S * N * kMaskBytes);
    if (L == 8) run<8>(a, &queue, S, gpf, wpb, blocks, act.data(), rew.data(), done.data(), ply.data(), mask.data());
    else if (L == 4) run<4>(a, &queue, S, gpf, wpb, blocks, act.data(), rew.data(), done.data(), ply.data(), mask.data());
    else if (L == 16) run<16>(a, &queue, S, gpf, wpb, blocks, act.data(), rew.data(), done.data(), ply.data(), mask.data());
    else run<32>(a, &queue, S, gpf, wpb, blocks, act.data(), rew.data(), done.data(), ply.data(), mask.data());
    dump(out + ".action", act.data(), act.size());
    dump(out + ".reward", rew.data(), rew.size());
    dump(out + ".done", done.data(), done.size());
    dump(out + ".ply", ply.data(), ply.size());
    dump(out + ".mask", mask.data(), mask.size());
    dump(out + ".stats", stats.data(), stats.size());
    std::printf("status %d %d\n", status[0], status[1]);
    return 0;
}
