// Parameters of CRYSTALS-Dilithium round 3 for the three NIST levels
// (Table 1 of arXiv 2211.12265) and the byte sizes of keys and signatures that
// follow from the round-3 encodings (little-endian bit streams).
#pragma once
#include <cstddef>
#include <cstdint>

namespace dil {

constexpr int N = 256;
constexpr int32_t Q = 8380417;
constexpr int D = 13;
// q^-1 mod 2^32, used by the signed Montgomery reduction (R = 2^32).
constexpr int32_t QINV = 58728449;

template <int LEVEL> struct Params;

template <> struct Params<2> {
    static constexpr int K = 4, L = 4, ETA = 2, TAU = 39, BETA = 78, OMEGA = 80;
    static constexpr int32_t GAMMA1 = 1 << 17, GAMMA2 = (Q - 1) / 88;
};
template <> struct Params<3> {
    static constexpr int K = 6, L = 5, ETA = 4, TAU = 49, BETA = 196, OMEGA = 55;
    static constexpr int32_t GAMMA1 = 1 << 19, GAMMA2 = (Q - 1) / 32;
};
template <> struct Params<5> {
    static constexpr int K = 8, L = 7, ETA = 2, TAU = 60, BETA = 120, OMEGA = 75;
    static constexpr int32_t GAMMA1 = 1 << 19, GAMMA2 = (Q - 1) / 32;
};

// Derived widths and sizes.
template <int LEVEL> struct Lv : Params<LEVEL> {
    using P = Params<LEVEL>;
    static constexpr int ZBITS = (P::GAMMA1 == (1 << 17)) ? 18 : 20;
    static constexpr int W1BITS = (P::GAMMA2 == (Q - 1) / 88) ? 6 : 4;
    static constexpr int ETABITS = (P::ETA == 2) ? 3 : 4;
    static constexpr int ALPHA = 2 * P::GAMMA2;
    static constexpr int M_HI = (Q - 1) / ALPHA;        // number of HighBits values
    static constexpr int POLYT1 = N * 10 / 8;           // 320
    static constexpr int POLYT0 = N * D / 8;            // 416
    static constexpr int POLYETA = N * ETABITS / 8;     // 96 or 128
    static constexpr int POLYZ = N * ZBITS / 8;         // 576 or 640
    static constexpr int POLYW1 = N * W1BITS / 8;       // 192 or 128
    static constexpr int PK = 32 + P::K * POLYT1;
    static constexpr int SK = 96 + (P::K + P::L) * POLYETA + P::K * POLYT0;
    static constexpr int SIG = 32 + P::L * POLYZ + P::OMEGA + P::K;
    // byte offsets inside sk: rho | K | tr | s1 | s2 | t0
    static constexpr int SK_S1 = 96;
    static constexpr int SK_S2 = 96 + P::L * POLYETA;
    static constexpr int SK_T0 = 96 + (P::K + P::L) * POLYETA;
    // byte offsets inside sig: c~ | z | h
    static constexpr int SIG_Z = 32;
    static constexpr int SIG_H = 32 + P::L * POLYZ;
    // nonce kappa + i (i < l) must fit 16 bits; kappa = l * iteration
    static constexpr int MAX_ITER = (65536 - P::L) / P::L + 1;
};

}  // namespace dil
