// Host-side plan: Algorithm 1 Steps I-II and the constants of the exact CRT.
//
// Step I   moduli p_l <= 256, pairwise coprime.  The paper does not list them;
//          this library takes the greedy descending set (keep c = 256, 255,
//          ... when coprime to all kept so far).
// Step II  q_l = (P/p_l)^-1 mod p_l, CRT weights w_l = (P/p_l) q_l, so that
//          sum_l w_l E'_l == A'B' (mod P) (Section II).
// The CRT is evaluated exactly in L 32-bit limbs modulo 2^(32L) (2^(32L-1) > 2P):
//   c' = sum_l w_l u_l + r' (2^(32L) - P) + K,  u_l = v_l + o,
//   r' = r + R0 with r = round(S/P) and K = R0 P - o sum_l w_l,
// where v_l is any integer congruent to c' modulo p_l: E'_l for real input
// (o = 128, K), and the unreduced Karatsuba combinations D_l - E_l (o = 255,
// KR) and F_l - D_l - E_l (o = 382, KI) for complex input.
#include <cmath>
#include <cstring>
#include <mutex>

#include "emu_internal.h"

namespace emu {
namespace {

constexpr int kBigLimbs = 8;  // 256-bit scratch integers

struct Big {
  uint32_t v[kBigLimbs];
  Big() { std::memset(v, 0, sizeof(v)); }
  explicit Big(uint64_t x) : Big() {
    v[0] = static_cast<uint32_t>(x);
    v[1] = static_cast<uint32_t>(x >> 32);
  }
};

void mul_small(Big& a, uint32_t s) {
  uint64_t carry = 0;
  for (int i = 0; i < kBigLimbs; ++i) {
    uint64_t t = static_cast<uint64_t>(a.v[i]) * s + carry;
    a.v[i] = static_cast<uint32_t>(t);
    carry = t >> 32;
  }
}

uint32_t divmod_small(Big& a, uint32_t s) {  // a /= s, returns a mod s
  uint64_t rem = 0;
  for (int i = kBigLimbs - 1; i >= 0; --i) {
    uint64_t cur = (rem << 32) | a.v[i];
    a.v[i] = static_cast<uint32_t>(cur / s);
    rem = cur % s;
  }
  return static_cast<uint32_t>(rem);
}

void add(Big& a, const Big& b) {
  uint64_t carry = 0;
  for (int i = 0; i < kBigLimbs; ++i) {
    uint64_t t = static_cast<uint64_t>(a.v[i]) + b.v[i] + carry;
    a.v[i] = static_cast<uint32_t>(t);
    carry = t >> 32;
  }
}

void sub(Big& a, const Big& b) {  // modulo 2^256
  int64_t borrow = 0;
  for (int i = 0; i < kBigLimbs; ++i) {
    int64_t t = static_cast<int64_t>(a.v[i]) - b.v[i] - borrow;
    borrow = t < 0 ? 1 : 0;
    a.v[i] = static_cast<uint32_t>(t);
  }
}

int bitlen(const Big& a) {
  for (int i = kBigLimbs - 1; i >= 0; --i)
    if (a.v[i]) return 32 * i + (32 - __builtin_clz(a.v[i]));
  return 0;
}

void shl(Big& a, int s) {
  Big r;
  int w = s / 32, b = s % 32;
  for (int i = kBigLimbs - 1; i >= 0; --i) {
    if (i - w < 0) continue;
    uint64_t x = static_cast<uint64_t>(a.v[i - w]) << b;
    if (b && i - w - 1 >= 0) x |= a.v[i - w - 1] >> (32 - b);
    r.v[i] = static_cast<uint32_t>(x);
  }
  a = r;
}

uint64_t extract64(const Big& a, int s) {  // floor(a / 2^s) truncated to 64 bits
  uint64_t r = 0;
  for (int bit = 63; bit >= 0; --bit) {
    int pos = s + bit;
    if (pos < 32 * kBigLimbs && ((a.v[pos / 32] >> (pos % 32)) & 1u)) r |= (1ull << bit);
  }
  return r;
}

// Round a non-negative integer to the nearest double (ties to even).
double big_to_double(const Big& a) {
  const int b = bitlen(a);
  if (b == 0) return 0.0;
  if (b <= 64) {
    uint64_t v = extract64(a, 0);
    if (b <= 53) return static_cast<double>(v);
    // round the 64-bit value: the conversion is RN
    return static_cast<double>(v);
  }
  const int sh = b - 64;
  uint64_t top = extract64(a, sh);
  bool sticky = false;
  for (int i = 0; i < sh; ++i)
    if ((a.v[i / 32] >> (i % 32)) & 1u) sticky = true;
  if (sticky) top |= 1u;                   // the 11 extra bits below the 53 keep the rounding correct
  return std::ldexp(static_cast<double>(top), sh);
}

// Exact difference a - b of a non-negative Big and a double holding an integer, as a double (RN).
double big_minus_double(const Big& a, double d) {
  // d is an integer-valued double >= 0 with at most 53 significant bits
  int e;
  const double f = std::frexp(d, &e);                   // d = f 2^e, 0.5 <= f < 1
  const uint64_t mant = static_cast<uint64_t>(std::ldexp(f, 53));
  const int sh = e - 53;
  Big bd(mant);
  if (sh > 0) shl(bd, sh);
  // compare a and bd
  bool a_ge = true;
  for (int i = kBigLimbs - 1; i >= 0; --i)
    if (a.v[i] != bd.v[i]) {
      a_ge = a.v[i] > bd.v[i];
      break;
    }
  Big diff = a_ge ? a : bd;
  sub(diff, a_ge ? bd : a);
  const double r = big_to_double(diff);
  return a_ge ? r : -r;
}

// IEEE binary16 bits of x rounded to nearest (ties to even), |x| < 65504, and back.
uint16_t half_bits(double x) {
  const uint16_t sign = x < 0 ? 0x8000u : 0u;
  x = std::fabs(x);
  if (x == 0.0) return sign;
  int e;
  std::frexp(x, &e);                               // x = f 2^e, 0.5 <= f < 1: leading bit 2^(e-1)
  int lsb = (e - 1) - 10;                          // exponent of the last kept bit
  if (lsb < -24) lsb = -24;                        // subnormal range
  double mant = std::nearbyint(std::ldexp(x, -lsb));
  if (mant >= 2048.0) {                            // rounding carried into the next binade
    mant /= 2.0;
    ++lsb;
  }
  if (mant < 1024.0) return static_cast<uint16_t>(sign | static_cast<uint16_t>(mant));   // subnormal
  return static_cast<uint16_t>(sign | ((lsb + 25) << 10) | (static_cast<uint16_t>(mant) - 1024u));
}

double half_value(uint16_t h) {
  const int ex = (h >> 10) & 0x1F;
  const double mant = ex ? (1024 + (h & 0x3FF)) : (h & 0x3FF);
  const double v = std::ldexp(mant, ex ? ex - 25 : -24);
  return (h & 0x8000u) ? -v : v;
}

int gcd_int(int a, int b) {
  while (b) {
    int t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace
int plan_exponent(const Plan& pl, uint64_t S);
namespace {

void build(int N, Plan& pl) {
  std::memset(&pl, 0, sizeof(pl));
  pl.N = N;
  // Step I: greedy descending pairwise-coprime moduli
  int count = 0;
  for (int c = 256; c >= 2 && count < N; --c) {
    bool ok = true;
    for (int i = 0; i < count; ++i)
      if (gcd_int(c, pl.p[i]) != 1) ok = false;
    if (ok) pl.p[count++] = c;
  }
  Big P(1);
  for (int l = 0; l < N; ++l) mul_small(P, static_cast<uint32_t>(pl.p[l]));
  const int bitsP = bitlen(P);
  // limbs hold c' + {-P, 0, P} with |c'| <= P/2 (accurate mode) in two's complement: 2^(32L-1) > 2P
  pl.L = (bitsP + 2 + 31) / 32;
  // Step II and the CRT weights
  Big sumw;
  double sum_qp = 0.0;                         // sum_l q_l / p_l = sum_l w_l / P
  uint32_t qs[kMaxModuli] = {};
  for (int l = 0; l < N; ++l) {
    const uint32_t p = static_cast<uint32_t>(pl.p[l]);
    Big M = P;
    divmod_small(M, p);                        // M = P / p_l exactly
    Big Mc = M;
    const uint32_t mmod = divmod_small(Mc, p);  // (P/p_l) mod p_l
    uint32_t q = 0;
    for (uint32_t t = 1; t < p; ++t)            // inverse by exhaustive search
      if ((mmod * t) % p == 1u) {
        q = t;
        break;
      }
    qs[l] = q;
    Big w = M;
    mul_small(w, q);
    for (int t = 0; t < kMaxLimbs; ++t) pl.w[l][t] = t < pl.L ? w.v[t] : 0u;
    add(sumw, w);
    sum_qp += static_cast<double>(q) / static_cast<double>(p);
    pl.barrett[l] = static_cast<uint32_t>((1ull << 32) / p);
    pl.two32[l] = static_cast<uint32_t>((1ull << 32) % p);
    uint32_t v = 1 % p;
    for (int s = 0; s < kPow2Table; ++s) {
      pl.pow2[l][s] = static_cast<uint8_t>(v);
      v = (v * 2u) % p;
    }
    for (int t = 0; t < kMaxChunks; ++t) {
      const int e = kChunkBits * t;           // 2^e mod p, then symmetric
      const int r = e < kPow2Table ? pl.pow2[l][e] : 0;
      const int sr = 2 * r >= static_cast<int>(p) ? r - static_cast<int>(p) : r;
      pl.w13[l][t] = static_cast<float>(sr);
    }
    pl.inv_p[l] = static_cast<float>(1.0 / static_cast<double>(p));
  }
  // the paper's floating-point CRT: s1 on the grid 2^g, s2 = RN(w - s1)
  {
    int cl = 0;
    while ((1 << cl) < N) ++cl;                                 // ceil(log2 N)
    const int g = bitsP - (46 - cl);
    for (int l = 0; l < N; ++l) {
      Big w;
      for (int t = 0; t < kMaxLimbs; ++t) w.v[t] = pl.w[l][t];
      // w itself may need more limbs than L stores: recompute from P
      w = P;
      divmod_small(w, static_cast<uint32_t>(pl.p[l]));
      uint32_t q = 0;
      {
        Big Mc = w;
        const uint32_t mmod = divmod_small(Mc, static_cast<uint32_t>(pl.p[l]));
        for (uint32_t t = 1; t < static_cast<uint32_t>(pl.p[l]); ++t)
          if ((mmod * t) % static_cast<uint32_t>(pl.p[l]) == 1u) {
            q = t;
            break;
          }
      }
      mul_small(w, q);
      Big hi = w;
      if (g > 0) {
        // hi = floor(w / 2^g) 2^g
        for (int i = 0; i < g; ++i) hi.v[i / 32] &= ~(1u << (i % 32));
      }
      pl.s1[l] = big_to_double(hi);                             // <= 46 significant bits: exact
      pl.s2[l] = big_minus_double(w, pl.s1[l]);
      pl.wd[l] = big_to_double(w);
    }
    pl.Ph = big_to_double(P);
    pl.Pl = big_minus_double(P, pl.Ph);
  }
  // the CRT quotient estimate from the accumulated limbs: sum_t acc_t 2^(32 t) / P,
  // less the offset the unsigned residues carry (u = E' + 128, D - E + 255, F - D - E + 382)
  for (int t = 0; t < kMaxLimbs; ++t)
    pl.qinv[t] = t < pl.L ? static_cast<float>(std::ldexp(1.0, 32 * t) / pl.Ph) : 0.0f;
  pl.off128 = static_cast<float>(128.0 * sum_qp);
  pl.off255 = static_cast<float>(255.0 * sum_qp);
  pl.off382 = static_cast<float>(382.0 * sum_qp);
  // negP = 2^(32L) - P, K = R0 P - 128 sum w (mod 2^(32L))
  Big zero;
  Big negP = zero;
  sub(negP, P);
  pl.R0 = 384 * N;                             // r >= -383 N for every offset below
  auto offset_const = [&](uint32_t o) {        // R0 P - o sum w
    Big Kc = P;
    mul_small(Kc, static_cast<uint32_t>(pl.R0));
    Big wo = sumw;
    mul_small(wo, o);
    sub(Kc, wo);
    return Kc;
  };
  const Big K = offset_const(128u), KR = offset_const(255u), KI = offset_const(382u);
  Big H = P;                                   // (P - 1) / 2
  sub(H, Big(1));
  divmod_small(H, 2u);
  for (int t = 0; t < kMaxLimbs; ++t) {
    pl.negP[t] = t < pl.L ? negP.v[t] : 0u;
    pl.K[t] = t < pl.L ? K.v[t] : 0u;
    pl.KR[t] = t < pl.L ? KR.v[t] : 0u;
    pl.KI[t] = t < pl.L ? KI.v[t] : 0u;
    pl.Pw[t] = t < pl.L ? P.v[t] : 0u;
    pl.H[t] = t < pl.L ? H.v[t] : 0u;
  }
  // tensor-core CRT constants
  {
    Big mask;                                  // 2^(32L) - 1
    for (int t = 0; t < pl.L; ++t) mask.v[t] = 0xFFFFFFFFu;
    for (int v = 0; v < 2; ++v) {
      const int b = v == 0 ? 10 : 9;
      for (int c = 0; c < kTcDigits; ++c) pl.tcmul[v][c] = 1u << ((b * c) & 31);
      for (int l = 0; l < N; ++l) {
        // balanced base-2^b digits of w_l (w_l < P: a few digits more than bitlen(P) / b at most)
        Big w;
        for (int t = 0; t < kMaxLimbs; ++t) w.v[t] = pl.w[l][t];
        int64_t carry = 0;
        for (int c = 0; c < kTcDigits; ++c) {
          // digit = (w >> bc) mod 2^b + carry, balanced into [-2^(b-1), 2^(b-1))
          int64_t d = static_cast<int64_t>(extract64(w, b * c) & ((1ull << b) - 1)) + carry;
          carry = 0;
          if (d >= (int64_t(1) << (b - 1))) {
            d -= int64_t(1) << b;
            carry = 1;
          }
          pl.tcdig[v][l][c] = static_cast<int16_t>(d);
        }
      }
    }
    // w_l / P = q_l / p_l as hi + lo in fp16 (the quotient estimate's columns)
    for (int l = 0; l < N; ++l) {
      const double g = static_cast<double>(qs[l]) / static_cast<double>(pl.p[l]);
      const uint16_t hi = half_bits(g);
      pl.tcest[l][0] = hi;
      pl.tcest[l][1] = half_bits(g - half_value(hi));
    }
    // K for each layout: R0 P - magic * sum over its digit slots that land below 2^(32L)
    const int slots[3] = {14, 30, 30}, bases[3] = {10, 9, 10};
    for (int v = 0; v < 3; ++v) {
      Big bias;
      for (int c = 0; c < slots[v]; ++c) {
        const int bit = bases[v] * c;
        if (bit >= 32 * pl.L) continue;
        Big term(0x4B400000ull);
        shl(term, bit);
        add(bias, term);
      }
      Big Kc = P;
      mul_small(Kc, static_cast<uint32_t>(pl.R0));
      sub(Kc, bias);
      for (int t = 0; t < kMaxLimbs; ++t) pl.tcK[v][t] = t < pl.L ? Kc.v[t] : 0u;
    }
  }
  // X = (P - 1) 2^27 for the fast-mode exponent rule
  Big X = P;
  sub(X, Big(1));
  shl(X, 27);
  const int bx = bitlen(X);
  pl.sX = bx > 63 ? bx - 63 : 0;
  pl.Xtop = extract64(X, pl.sX);
  // the largest exponent E (S at its minimum) bounds every |a'| < 2^(E+1)
  const int Emax = plan_exponent(pl, 0);
  pl.nchunk = (Emax + 1 + kChunkBits - 1) / kChunkBits;
  if (pl.nchunk < 1) pl.nchunk = 1;
  // accurate mode: |a'| < 64 * 2^E with E at most its value for a bound of 1
  const int Eaccu = plan_exponent_accu(pl, 1);
  pl.nchunk_accu = (Eaccu + 6 + kChunkBits - 1) / kChunkBits;
  if (pl.nchunk_accu < 1) pl.nchunk_accu = 1;
}

std::mutex g_mu;
Plan g_plans[kMaxModuli + 1];
bool g_built[kMaxModuli + 1] = {};

}  // namespace

const Plan* get_plan(int N) {
  if (N < EMU_MIN_MODULI || N > EMU_MAX_MODULI) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_built[N]) {
    build(N, g_plans[N]);
    g_built[N] = true;
  }
  return &g_plans[N];
}

// Largest E with 4^E * M <= X, X = (P-1) 2^27 = Xtop 2^sX + rest, for M >= 1.
// Shared by host queries; the device copy lives in k_scale.cu.
int exponent_le(const Plan& pl, uint64_t M) {
  const int bm = 64 - __builtin_clzll(M);
  const int bx = pl.sX + (64 - __builtin_clzll(pl.Xtop));
  auto fits = [&](int E) -> bool {
    const int sh = 2 * E - pl.sX;            // floor(X / 4^E) = floor(Xtop * 2^-sh)
    if (sh >= 64) return false;
    if (sh >= 0) return M <= (pl.Xtop >> sh);
    if (-sh >= 64) return true;
    const unsigned __int128 lhs = static_cast<unsigned __int128>(pl.Xtop) << (-sh);
    return static_cast<unsigned __int128>(M) <= lhs;
  };
  int d = bx - bm;
  int E = d >= 0 ? d / 2 : -((-d + 1) / 2);   // floor(d / 2)
  while (!fits(E)) --E;
  while (fits(E + 1)) ++E;
  return E;
}

// Fast mode: largest E with 4^E * max(2^32, S) <= (P-1) 2^27.
int plan_exponent(const Plan& pl, uint64_t S) { return exponent_le(pl, S > (1ull << 32) ? S : (1ull << 32)); }

// Accurate mode: largest E with 4^E * max(M, 1) <= (P-1)/2, i.e. 4^E max(M,1) 2^28 <= X.
int plan_exponent_accu(const Plan& pl, uint64_t M) { return exponent_le(pl, (M > 1 ? M : 1ull) << 28); }

}  // namespace emu

extern "C" {

emu_status_t emu_plan_info(int num_moduli, int32_t* moduli, int32_t* q, uint32_t* p_limbs,
                           int32_t* crt_limbs) {
  const emu::Plan* pl = emu::get_plan(num_moduli);
  if (!pl) return EMU_ERR_MODULI_RANGE;
  emu::Big P(1);
  for (int l = 0; l < pl->N; ++l) {
    if (moduli) moduli[l] = pl->p[l];
    emu::mul_small(P, static_cast<uint32_t>(pl->p[l]));
  }
  if (q) {
    for (int l = 0; l < pl->N; ++l) {
      emu::Big M = P;
      emu::divmod_small(M, static_cast<uint32_t>(pl->p[l]));
      emu::Big Mc = M;
      const uint32_t mmod = emu::divmod_small(Mc, static_cast<uint32_t>(pl->p[l]));
      int32_t qq = 0;
      for (int t = 1; t < pl->p[l]; ++t)
        if ((mmod * static_cast<uint32_t>(t)) % static_cast<uint32_t>(pl->p[l]) == 1u) {
          qq = t;
          break;
        }
      q[l] = qq;
    }
  }
  if (p_limbs)
    for (int t = 0; t < 8; ++t) p_limbs[t] = P.v[t];
  if (crt_limbs) *crt_limbs = pl->L;
  return EMU_OK;
}

int emu_plan_exponent(int num_moduli, uint64_t S) {
  const emu::Plan* pl = emu::get_plan(num_moduli);
  if (!pl) return -100000;
  return emu::plan_exponent(*pl, S);
}

int emu_plan_exponent_accu(int num_moduli, uint64_t M) {
  const emu::Plan* pl = emu::get_plan(num_moduli);
  if (!pl || M >= (1ull << 35)) return -100000;
  return emu::plan_exponent_accu(*pl, M);
}

}  // extern "C"
