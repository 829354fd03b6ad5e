/*
 * Oracle observation planes (App. C, "Information State Representation"):
 * 487 channels of 10x10 for one player, in the absolute board frame.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Channel map (App. C.1-C.2; readings marked *):
 *   0-11    own piece of type T
 *   12-23   P(opponent piece here has type T) under uniform setup and moves
 *   24-35   the same for own pieces, from the opponent's side
 *   36/37   own / opponent unrevealed piece        38 empty square (lakes 0)
 *   39/40   own / opponent piece that has moved
 *   41      ply / max_plies *(whole plane)         42 battleless / k *(whole plane)
 *   43-52/53  own piece threatened a revealed rank / a hidden piece
 *   54-63/64  own piece evaded a revealed rank / a hidden threatener
 *   65-74/75  own piece was actively adjacent to a revealed rank / hidden piece
 *   76-108  channels 43-75 for opponent pieces
 *   109-119 / 120-130  own / opponent captured piece of type Spy..Marshal,Bomb,
 *           shown on its start square
 *   131-190 own piece of rank Spy..Marshal died here by cause 1-6:
 *           131 + 10*(cause-1) + rank index *(10 types per cause, Bomb dropped)
 *   191-250 the same for opponent pieces
 *   251-302 own protection planes (protected / protected against / was
 *           protected by / was protected against), 275, 288, 301 padding
 *   303-354 the same for opponent pieces *(the paper's "251-315" read as 251-302)
 *   355-454 one-hot start square of the occupant *(the paper's "355-455")
 *   455-486 the move played j+1 plies ago: destination +1, source -1
 *
 * Values: indicators are 0/1.  A probability or fraction num/den is stored as
 * uint8 floor(255*num/den + 1/2) and as the bf16 nearest (ties to even) to
 * the exact rational num/den.  -1 is uint8 255 and bf16 -1.0.
 *
 * Probabilities (channels 12-35), for the side whose pieces are estimated:
 *   R revealed pieces, S unrevealed pieces that moved more than one square
 *   (Scouts), M other unrevealed moved pieces, U unrevealed unmoved pieces.
 *   c_T = initial count - revealed or captured pieces of type T (- |S| for
 *   Scout); b = c_Flag + c_Bomb; m = sum of c_T over movable types.
 *   U piece: Bomb c_B/|U|, Flag c_F/|U|, movable T (|U|-b) c_T / (|U| m).
 *   M piece: movable T c_T/m.  S piece: Scout.  R piece: its type.
 *   These are the exact marginals of the uniform distribution over all type
 *   assignments consistent with the public history.
 */
#include <string.h>
#include "oracle.h"

static const int TYPE_COUNT[T_NTYPES] = { 1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6 };

uint8_t or_u8_ratio(uint32_t num, uint32_t den)
{
    return (uint8_t)((510u * num + den) / (2u * den));
}

/* bf16 bits nearest to num/den (ties to even); num/den in [0, 1]. */
uint16_t or_bf16_ratio(uint32_t num, uint32_t den)
{
    if (num == 0) return 0;
    uint64_t n = num, d = den;
    int e = 0;
    while (n < d) { n *= 2; e -= 1; }
    while (n >= 2 * d) { d *= 2; e += 1; }
    /* 1 <= n/d < 2: 8 significant bits */
    uint64_t q = (n * 128) / d;
    uint64_t rem = n * 128 - q * d;
    if (2 * rem > d || (2 * rem == d && (q & 1))) q += 1;
    if (q == 256) { q = 128; e += 1; }
    return (uint16_t)(((uint32_t)(e + 127) << 7) | (uint32_t)(q - 128));
}

/* num/den per (piece, type) for the pieces of `side`. */
static void marginals(const or_game* g, int side, uint32_t num[40][T_NTYPES], uint32_t den[40][T_NTYPES])
{
    int c[T_NTYPES];
    int nS = 0, nM = 0, nU = 0;
    for (int t = 0; t < T_NTYPES; ++t) c[t] = TYPE_COUNT[t];
    for (int k = 0; k < 40; ++k) {
        int p = side * 40 + k;
        if (!g->alive[p] || g->revealed[p]) { c[g->type[p]]--; continue; }
        if (g->scout_known[p]) nS++;
        else if (g->moved[p]) nM++;
        else nU++;
    }
    c[T_SCOUT] -= nS;
    int b = c[T_FLAG] + c[T_BOMB];
    int m = 0;
    for (int t = 0; t <= T_MARSHAL; ++t) m += c[t];
    for (int k = 0; k < 40; ++k) {
        int p = side * 40 + k;
        for (int t = 0; t < T_NTYPES; ++t) { num[k][t] = 0; den[k][t] = 1; }
        if (!g->alive[p]) continue;
        if (g->revealed[p]) { num[k][g->type[p]] = 1; continue; }
        if (g->scout_known[p]) { num[k][T_SCOUT] = 1; continue; }
        if (g->moved[p]) {
            for (int t = 0; t <= T_MARSHAL; ++t) { num[k][t] = (uint32_t)c[t]; den[k][t] = (uint32_t)m; }
            continue;
        }
        num[k][T_FLAG] = (uint32_t)c[T_FLAG]; den[k][T_FLAG] = (uint32_t)nU;
        num[k][T_BOMB] = (uint32_t)c[T_BOMB]; den[k][T_BOMB] = (uint32_t)nU;
        for (int t = 0; t <= T_MARSHAL; ++t) {
            if (m == 0) continue;
            num[k][t] = (uint32_t)((nU - b) * c[t]);
            den[k][t] = (uint32_t)(nU * m);
        }
    }
}

/* Public entry for tests: num/den of side's pieces, den as one array per type. */
void or_side_marginals(const or_game* g, int side, uint32_t* num /*[40][12]*/, uint32_t* den /*[40][12]*/)
{
    uint32_t n[40][T_NTYPES], d[40][T_NTYPES];
    marginals(g, side, n, d);
    memcpy(num, n, sizeof(n));
    memcpy(den, d, sizeof(d));
}

static void put(uint8_t* u8, uint16_t* bf, int ch, int s, int value)
{
    /* value: 1 or -1 */
    u8[ch * 100 + s] = value > 0 ? 1 : 255;
    bf[ch * 100 + s] = value > 0 ? 0x3F80 : 0xBF80;
}

static void put_ratio(uint8_t* u8, uint16_t* bf, int ch, int s, uint32_t num, uint32_t den)
{
    u8[ch * 100 + s] = or_u8_ratio(num, den);
    bf[ch * 100 + s] = or_bf16_ratio(num, den);
}

static void put_bits(uint8_t* u8, uint16_t* bf, int ch0, int s, uint32_t bits, int nbits, int skip)
{
    for (int i = 0; i < nbits; ++i)
        if ((bits >> i) & 1) put(u8, bf, ch0 + i + (i >= skip ? 1 : 0), s, 1);
}

void or_encode_planes(const or_game* g, int player, uint8_t* u8, uint16_t* bf)
{
    memset(u8, 0, OR_NCHAN * 100);
    memset(bf, 0, OR_NCHAN * 100 * sizeof(uint16_t));
    int opp = 1 - player;
    uint32_t num[2][40][T_NTYPES], den[2][40][T_NTYPES];
    marginals(g, 0, num[0], den[0]);
    marginals(g, 1, num[1], den[1]);

    for (int s = 0; s < OR_NSQ; ++s)
        if (g->board[s] == -1) put(u8, bf, 38, s, 1);
    for (int s = 0; s < OR_NSQ; ++s) {
        put_ratio(u8, bf, 41, s, (uint32_t)g->ply, (uint32_t)g->rules.max_plies);
        put_ratio(u8, bf, 42, s, (uint32_t)g->battleless, (uint32_t)g->rules.battleless_limit);
    }

    for (int p = 0; p < OR_NPIECE; ++p) {
        int side = p / 40, k = p % 40;
        int own = side == player;
        int start = side == 0 ? k : 60 + k;
        if (!g->alive[p]) {
            int t = g->type[p];
            int ti = t <= T_MARSHAL ? t : (t == T_BOMB ? 10 : -1);
            if (ti >= 0) put(u8, bf, (own ? 109 : 120) + ti, start, 1);
            if (t <= T_MARSHAL && g->cause[p] >= 1)
                put(u8, bf, (own ? 131 : 191) + 10 * (g->cause[p] - 1) + t, g->sq[p], 1);
            continue;
        }
        int s = g->sq[p];
        if (own) put(u8, bf, g->type[p], s, 1);
        /* probabilities: the opponent's pieces as seen by `player` go to 12-23,
           `player`'s own pieces as seen by the opponent go to 24-35 */
        int base = own ? 24 : 12;
        for (int t = 0; t < T_NTYPES; ++t)
            if (num[side][k][t]) put_ratio(u8, bf, base + t, s, num[side][k][t], den[side][k][t]);
        if (!g->revealed[p]) put(u8, bf, own ? 36 : 37, s, 1);
        if (g->moved[p]) put(u8, bf, own ? 39 : 40, s, 1);
        int fb = own ? 43 : 76;
        put_bits(u8, bf, fb, s, g->f_threat[p], 11, 99);
        put_bits(u8, bf, fb + 11, s, g->f_evade[p], 11, 99);
        put_bits(u8, bf, fb + 22, s, g->f_active[p], 11, 99);
        int pb = own ? 251 : 303;
        put_bits(u8, bf, pb, s, g->f_prot[p], 13, 99);          /* 251-263 */
        put_bits(u8, bf, pb + 13, s, g->f_pagainst[p], 12, 11);   /* 264-274, pad 275, 276 */
        put_bits(u8, bf, pb + 26, s, g->f_pby[p], 12, 11);        /* 277-287, pad 288, 289 */
        put_bits(u8, bf, pb + 39, s, g->f_pbyagainst[p], 12, 11); /* 290-300, pad 301, 302 */
        put(u8, bf, 355 + start, s, 1);
    }
    for (int j = 0; j < 32; ++j) {
        if (g->hist[j] == 0xFFFF) break;
        int f = g->hist[j] / 100, t = g->hist[j] % 100;
        put(u8, bf, 455 + j, t, 1);
        put(u8, bf, 455 + j, f, -1);
    }
    (void)opp;
}
