// features.cuh -- sticky per-piece history features of the information state
// (App. C.1: threats, evasions, active adjacency, protection moves) and a
// single-move legality test, for the replay kernels.
//
// Per piece two 64-bit words:
//   A: bits 0-10 threatened (revealed rank Spy..Marshal, or bit 10 hidden),
//      bits 11-21 evaded, bits 22-32 actively adjacent (same 11-bit layout);
//      A's bit i is channel 43+i for own pieces and 76+i for opponent pieces.
//   B: bits 0-51 in the order of channels 251-302 (own) / 303-354 (opponent):
//      0-10 protected a revealed Spy..Marshal,Bomb, 11 an empty square,
//      12 a hidden piece; 13-23 protected against a revealed type, 24 padding,
//      25 against a hidden piece; 26-36 was protected by a revealed type, 37
//      padding, 38 by a hidden piece; 39-49 was protected against a revealed
//      type, 50 padding, 51 against a hidden piece.
// Readings: a threat is a non-battle move ending next to enemy pieces; an
// evasion moves a piece that stood next to where the opponent's previous
// non-battle move ended to a square not next to it; active adjacency is an
// adjacent attack that was legal but not played; a protection answers a
// threat by moving another piece next to the threatened piece (or next to an
// empty square next to the threatener) from a square not next to it.
#pragma once
#include "engine.cuh"

namespace stg {

struct __align__(16) FeatSmem {
    uint64_t a[kPieces];
    uint64_t b[kPieces];
};

// 0-9 revealed rank, 10 hidden, -1 none (a revealed Bomb or Flag)
__device__ __forceinline__ int feat_rank_or_hidden(const SmemGame* G, int pid)
{
    if (!(G->c.flags[pid] & 2)) return 10;
    const int t = G->c.type[pid];
    return t <= kMarshal ? t : -1;
}
// 0-9 revealed rank, 10 revealed Bomb, `hidden` if hidden, -1 revealed Flag
__device__ __forceinline__ int feat_type11(const SmemGame* G, int pid, int hidden)
{
    if (!(G->c.flags[pid] & 2)) return hidden;
    const int t = G->c.type[pid];
    return t <= kMarshal ? t : (t == kBomb ? 10 : -1);
}
__device__ __forceinline__ uint64_t fbit(int i) { return i >= 0 ? (1ull << i) : 0ull; }

// Is action a legal for the player to move?  Warp-uniform.
__device__ __forceinline__ bool move_legal(const SmemGame* G, int a, uint32_t rule_flags, const uint16_t* ring,
                                           const uint64_t* pi)
{
    if (a < 0 || a >= 10000) return false;
    const int P = G->c.ply & 1;
    const int from = a / 100, to = a - 100 * (a / 100);
    const uint8_t X = G->board[from];
    if (X >= kPieces || (int)(X / 40) != P) return false;
    const int t = G->c.type[X];
    if (t >= kFlag) return false;
    if (to == from || is_lake(to)) return false;
    const uint8_t occ = G->board[to];
    if (occ < kPieces && (int)(occ / 40) == P) return false;
    const int fr = from / 10, fc = from - 10 * fr, tr = to / 10, tc = to - 10 * tr;
    if (fr != tr && fc != tc) return false;
    const int dist = abs(fr - tr) + abs(fc - tc);
    if (dist > 1) {
        if (t != kScout) return false;
        const int step = fr == tr ? (tc > fc ? 1 : -1) : (tr > fr ? 10 : -10);
        for (int q = from + step; q != to; q += step)
            if (G->board[q] != kEmpty) return false;
    }
    if ((rule_flags & kTwoSquare) && G->c.ts_pid[P] == X && G->c.ts_len[P] == 4 && two_square_blocks(G, P, to))
        return false;
    if ((rule_flags & kChase) && G->c.chaser == P && G->c.n_pi > 0 && occ == kEmpty) {
        const PlyCtx x = make_ctx(G);
        if (chase_blocks(G, x, pi, P, X, from, to)) return false;
    }
    return true;
}

// Active adjacency before action a: every own movable piece next to an
// enemy piece could have attacked it; those attacks other than the one
// played (and other than moves the two-square rule forbids) set the
// piece's bits 22-32.  Lane j handles from-squares 4j .. 4j+3 from the
// square sets (south, north, west, east neighbour is an enemy).  The bits
// are ORed in atomically: other warps may record features of the same ply.
__device__ __forceinline__ void active_adjacency(const SmemGame* G, FeatSmem* F, int a, uint32_t rule_flags)
{
    const int lane = threadIdx.x & 31;
    const int P = G->c.ply & 1;
    const bool ts_on = (rule_flags & kTwoSquare) && G->c.ts_pid[P] != kNone && G->c.ts_len[P] == 4;
    const Set128 mv{G->bmov[P][0] | G->bsco[P][0], G->bmov[P][1] | G->bsco[P][1]};
    const Set128 en = ld128(G->bocc[1 - P]);
    const Set128 nS = and128(mv, up10(en)), nN = and128(mv, dn10(en));
    const Set128 nW = and128(and128(mv, up1(en)), Set128{~kCol0Lo, ~kCol0Hi});
    const Set128 nE = and128(and128(mv, dn1(en)), Set128{~kCol9Lo, ~kCol9Hi});
    const int off = 4 * lane;
    const uint32_t bs = bits_at(nS, off, 4), bn = bits_at(nN, off, 4);
    const uint32_t bw = bits_at(nW, off, 4), be = bits_at(nE, off, 4);
    uint32_t any = bs | bn | bw | be;
    while (any) {
        const int c = __ffs(any) - 1;
        any &= any - 1;
        const int sq = off + c;
        const int pid = G->board[sq];
        uint64_t bits = 0;
#pragma unroll
        for (int dir = 0; dir < 4; ++dir) {
            const uint32_t m = dir == 0 ? bs : dir == 1 ? bn : dir == 2 ? bw : be;
            if (!((m >> c) & 1u)) continue;
            const int n = sq + (dir == 0 ? -10 : dir == 1 ? 10 : dir == 2 ? -1 : 1);
            if (sq * 100 + n == a) continue;
            if (ts_on && pid == G->c.ts_pid[P] && two_square_blocks(G, P, n)) continue;
            bits |= fbit(feat_rank_or_hidden(G, G->board[n])) << 22;
        }
        if (bits) atomicOr(reinterpret_cast<unsigned long long*>(&F->a[pid]), (unsigned long long)bits);
    }
    __syncwarp(0xFFFFFFFFu);
}

// Evasion and protection by action a (a non-battle move), from the position
// before it, on the calling warp's first lane: the mover evades the piece
// the opponent's previous non-battle move brought next to it (bits 11-21),
// or protects a piece that move threatens (B bits of the mover and the
// protected piece).  Atomic ORs as in active_adjacency.
__device__ __forceinline__ void evasion_protection(const SmemGame* G, FeatSmem* F, int a)
{
    const int lane = threadIdx.x & 31;
    const int P = G->c.ply & 1;
    const int from = a / 100, to = a - 100 * (a / 100);
    const int X = G->board[from];
    const bool battle = G->board[to] != kEmpty;
    if (lane == 0 && !battle) {
        unsigned long long* fa = reinterpret_cast<unsigned long long*>(F->a);
        unsigned long long* fb = reinterpret_cast<unsigned long long*>(F->b);
        const PlyCtx x = make_ctx(G);
        const int ap = x.prev_to;
        if (ap >= 0 && x.prev_nb && enemy_of(G->board[ap], P)) {
            const int A = G->board[ap];
            if (adjacent(from, ap) && !adjacent(to, ap))
                atomicOr(&fa[X], (unsigned long long)(fbit(feat_rank_or_hidden(G, A)) << 11));
            const int ar = ap / 10, ac = ap - 10 * ar;
            int nb[4], nn = 0;
            if (ar > 0 && !is_lake(ap - 10)) nb[nn++] = ap - 10;
            if (ar < 9 && !is_lake(ap + 10)) nb[nn++] = ap + 10;
            if (ac > 0 && !is_lake(ap - 1)) nb[nn++] = ap - 1;
            if (ac < 9 && !is_lake(ap + 1)) nb[nn++] = ap + 1;
            bool threatened = false;
            for (int i = 0; i < nn; ++i) {
                const uint8_t q = G->board[nb[i]];
                threatened |= q < kPieces && (int)(q / 40) == P;
            }
            if (threatened) {
                const int a_idx = feat_type11(G, A, 11);
                for (int i = 0; i < nn; ++i) {
                    const int s = nb[i];
                    const uint8_t B = G->board[s];
                    if (B < kPieces && ((int)(B / 40) != P || B == X)) continue;
                    if (!(adjacent(to, s) && !adjacent(from, s))) continue;
                    uint64_t bx = B == kEmpty ? fbit(11) : fbit(feat_type11(G, B, 12));
                    if (a_idx >= 0) bx |= fbit(a_idx == 11 ? 25 : 13 + a_idx);
                    atomicOr(&fb[X], (unsigned long long)bx);
                    if (B < kPieces) {
                        const int c_idx = feat_type11(G, X, 11);
                        uint64_t bb = 0;
                        if (c_idx >= 0) bb |= fbit(c_idx == 11 ? 38 : 26 + c_idx);
                        if (a_idx >= 0) bb |= fbit(a_idx == 11 ? 51 : 39 + a_idx);
                        atomicOr(&fb[B], (unsigned long long)bb);
                    }
                }
            }
        }
    }
    __syncwarp(0xFFFFFFFFu);
}

// Threats made by action a (a non-battle move ending next to enemy pieces),
// read from the position before the move: a non-battle move changes only
// its two squares (`from` holds the mover's own piece before the move and
// nothing after, neither an enemy of the mover) and no piece's flags, so a
// warp can record them while another warp works out the move.
__device__ __forceinline__ void threats_of_move(const SmemGame* G, FeatSmem* F, int a, bool battle)
{
    if ((threadIdx.x & 31) == 0 && !battle) {
        const int from = a / 100, to = a - 100 * (a / 100);
        const int X = G->board[from];
        const int P = X / 40;
        const int r = to / 10, c = to - 10 * r;
        uint64_t bits = 0;
        if (r > 0 && enemy_of(G->board[to - 10], P)) bits |= fbit(feat_rank_or_hidden(G, G->board[to - 10]));
        if (r < 9 && enemy_of(G->board[to + 10], P)) bits |= fbit(feat_rank_or_hidden(G, G->board[to + 10]));
        if (c > 0 && enemy_of(G->board[to - 1], P)) bits |= fbit(feat_rank_or_hidden(G, G->board[to - 1]));
        if (c < 9 && enemy_of(G->board[to + 1], P)) bits |= fbit(feat_rank_or_hidden(G, G->board[to + 1]));
        if (bits) atomicOr(reinterpret_cast<unsigned long long*>(&F->a[X]), (unsigned long long)bits);
    }
    __syncwarp(0xFFFFFFFFu);
}

}  // namespace stg
