// Test harness only: runs the observation kernels (k_replay, then
// k_obs_emit) on host threads through include/cuda_runtime.h of this
// directory, on inputs read from <in>.{setups,actions,game,ply,player}
// (player may be absent), and writes <out>.{planes,bf16,mask,status}.
//   obs_on_host in num_logs log_len B items_per_block out
#include <sys/stat.h>
#include "host_launch.h"
#include "obs_dev.cu"

int main(int argc, char** argv)
{
    const std::string in = argv[1], out = argv[6];
    const int num_logs = std::atoi(argv[2]), log_len = std::atoi(argv[3]), B = std::atoi(argv[4]);
    const int ipw = std::atoi(argv[5]);
    auto setups = load<uint8_t>(in + ".setups");
    auto actions = load<int16_t>(in + ".actions");
    auto game = load<int32_t>(in + ".game");
    auto ply = load<int16_t>(in + ".ply");
    struct stat st;
    std::vector<int8_t> player;
    if (stat((in + ".player").c_str(), &st) == 0) player = load<int8_t>(in + ".player");
    if ((int)setups.size() != 80 * num_logs || (int)actions.size() != num_logs * log_len || (int)game.size() != B ||
        (int)ply.size() != B || (!player.empty() && (int)player.size() != B)) {
        std::fprintf(stderr, "input sizes\n");
        return 2;
    }
    const st_rules rules{100, 1000, ST_RULE_TWO_SQUARE | ST_RULE_CHASE};
    std::vector<ItemState> items((size_t)B);
    std::vector<uint8_t> mask((size_t)B * kMaskBytes), status((size_t)B, 0xEE);
    std::vector<uint8_t> planes((size_t)B * kPlaneBytes, 0xAB);
    std::vector<uint16_t> bf((size_t)B * kPlaneBytes, 0xABAB);
    ReplayArgs a = replay_args(setups.data(), actions.data(), log_len, num_logs, game.data(), ply.data(), B, &rules);
    a.items_per_block = ipw;
    a.state_out = items.data();
    a.mask_out = mask.data();
    a.status = status.data();
    launch((B + ipw - 1) / ipw, 32 * kReplayWarps, sizeof(ReplaySmem), [=] { k_replay(a); });
    EmitArgs e{};
    e.items = items.data(); e.status = status.data(); e.player = player.empty() ? nullptr : player.data();
    e.B = B; e.R = a.R; e.planes = planes.data(); e.planes_bf16 = bf.data();
    launch((B + kEmitWarps - 1) / kEmitWarps, 32 * kEmitWarps, kEmitWarps * sizeof(EmitSmem), [=] { k_obs_emit(e); });
    dump(out + ".planes", planes.data(), planes.size());
    dump(out + ".bf16", bf.data(), bf.size());
    dump(out + ".mask", mask.data(), mask.size());
    dump(out + ".status", status.data(), status.size());
    std::printf("done\n");
    return 0;
}
