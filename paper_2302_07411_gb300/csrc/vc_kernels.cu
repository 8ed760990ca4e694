// vc_kernels.cu -- sm_103a kernels of the chaotic video cipher.
//
//   k_tables_*        subframe partition tables (pi_i, start bitmap, ranks, tile limits)
//   k_key_schedule    Alg. 1: PRBG_m keyed by K -> parameters P_m of every PRBG_a^i
//   k_frame_sc        Alg. 1: one confusion seed s_c per frame from PRBG_m
//   k_kmod            Eq. 1: shift table k(alpha) = floor(s_c sin(2 pi alpha / H)), reduced mod W
//   k_keystream       Sec. 3 + Alg. 2: r * S_i bytes per frame from every PRBG_a^i (Eq. 5 / Eq. 6)
//   k_enc_round       Eq. 1 (confusion) fused with Eq. 3 (diffusion) for one round
//   k_enc_fixup       completes the diffusion chains that cross row-band tiles
//   k_dec_round       Eq. 4 (inverse diffusion) fused with Eq. 2 (inverse confusion)
//
// Layout of a frame: H x W x C bytes, HWC.  Byte q of a frame belongs to pixel
// q / C; subframe i owns bytes [C pi_i, C pi_{i+1}), pi_i = floor(i P / n).
#include <cstdint>

#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "vc_internal.h"
#include "vc_maps.cuh"

namespace vc {

// cudaFuncSetAttribute(func, MaxDynamicSharedMemorySize, bytes) only when a
// kernel needs more than it was last allowed on the current device (the call
// costs host time on every launch otherwise).
static std::mutex g_smem_mu;
static std::map<std::pair<int, const void*>, int> g_smem_allowed;

template <typename K>
static cudaError_t allow_smem(K* func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_pair(dev, reinterpret_cast<const void*>(func));
  {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    auto it = g_smem_allowed.find(key);
    if (it != g_smem_allowed.end() && it->second >= bytes) return cudaSuccess;
  }
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    int& v = g_smem_allowed[key];
    if (bytes > v) v = bytes;
  }
  return e;
}

// =============================================================================
// Partition tables
// =============================================================================

__global__ void k_tables_pi(Layout L, int* pi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= L.n) pi[i] = (int)(((long long)i * L.P) / L.n);
}

__global__ void k_tables_bits(Layout L, const int* pi, uint32_t* sbits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L.n) {
    const int p = pi[i];
    atomicOr(&sbits[p >> 5], 1u << (p & 31));
  }
}

// srank[w] = #{i < n : pi_i < 32 w} = min(n, ceil(32 w n / P)).
__global__ void k_tables_rank(Layout L, int* srank, int nwords) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < nwords) {
    const long long x = 32LL * w;
    const long long r = (x * L.n + L.P - 1) / L.P;
    srank[w] = (int)(r < L.n ? r : L.n);
  }
}

// fixlim[s] = first subframe-start byte >= the first byte of sub-tile s (rows
// [s R, (s + 1) R)), capped at its end: the smallest i with pi_i >= x0 is
// ceil(x0 n / P).
__global__ void k_tables_fixlim(Layout L, int* fixlim) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < L.NS) {
    const long long x0 = (long long)t * L.R * L.W;
    const long long istar = (x0 * L.n + L.P - 1) / L.P;
    const int rows_end = min(L.H, (t + 1) * L.R);
    long long fl = (long long)rows_end * L.W * L.C;
    if (istar < L.n) {
      const long long ps = (istar * L.P) / L.n;
      if (ps * L.C < fl) fl = ps * L.C;
    }
    fixlim[t] = (int)fl;
  }
}

cudaError_t launch_build_tables(const Layout& L, int* pi, uint32_t* sbits, int* srank, int* fixlim, cudaStream_t st) {
  const int nwords = L.P / 32 + 2;
  cudaError_t e = cudaMemsetAsync(sbits, 0, sizeof(uint32_t) * nwords, st);
  if (e != cudaSuccess) return e;
  k_tables_pi<<<(L.n + 1 + 255) / 256, 256, 0, st>>>(L, pi);
  k_tables_bits<<<(L.n + 255) / 256, 256, 0, st>>>(L, pi, sbits);
  k_tables_rank<<<(nwords + 255) / 256, 256, 0, st>>>(L, srank, nwords);
  k_tables_fixlim<<<(L.NS + 255) / 256, 256, 0, st>>>(L, fixlim);
  return cudaGetLastError();
}

// =============================================================================
// PRBG_m (Alg. 1): key schedule and per-frame confusion seeds
// =============================================================================

// Next 6-byte group U of PRBG_m's byte stream (first byte least significant).
__device__ uint64_t main_next_group(MainPrbg& m) {
  if (m.carry_len == 0) {
    if (m.kind == 0) {  // PLCM pair, 6 bytes per iterate
      m.s[0] = plcm_step(m.s[0], m.s[1], __dsub_rn(0.5, m.s[1]));
      m.s[2] = plcm_step(m.s[2], m.s[3], __dsub_rn(0.5, m.s[3]));
      m.carry[0] = mant48(m.s[0]) ^ mant48(m.s[2]);
      m.carry[1] = 0;
      m.carry_len = 6;
    } else if (m.kind == 2) {  // logistic pair, 6 bytes per iterate
      m.s[0] = logistic_step(m.s[0], m.s[1]);
      m.s[2] = logistic_step(m.s[2], m.s[3]);
      m.carry[0] = mant48(m.s[0]) ^ mant48(m.s[2]);
      m.carry[1] = 0;
      m.carry_len = 6;
    } else {  // single 2DLASM, x bytes then y bytes
      lasm_step(m.s[0], m.s[1], __dmul_rn(kPi, m.s[2]));
      const uint64_t vx = mant48(m.s[0]), vy = mant48(m.s[1]);
      m.carry[0] = vx | (vy << 48);
      m.carry[1] = vy >> 16;
      m.carry_len = 12;
    }
  }
  const uint64_t U = m.carry[0] & 0xFFFFFFFFFFFFull;
  m.carry[0] = (m.carry[0] >> 48) | (m.carry[1] << 16);
  m.carry[1] >>= 48;
  m.carry_len -= 6;
  return U;
}

// u = (U + 1/2) 2^-48, exact.
__device__ __forceinline__ double unit_of(uint64_t U) { return __dmul_rn(__ull2double_rn(2 * U + 1), 0x1p-49); }

__global__ void k_key_schedule(int kind, MainPrbg* mp, Chains ch, int n) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  MainPrbg m = *mp;
  for (int i = 0; i < n; i++) {
    if (kind == 0) {
      const double u1 = unit_of(main_next_group(m));
      const double u2 = unit_of(main_next_group(m));
      const double u3 = unit_of(main_next_group(m));
      const double u4 = unit_of(main_next_group(m));
      const double p1 = __dadd_rn(0.05, __dmul_rn(0.4, u2));
      const double p2 = __dadd_rn(0.05, __dmul_rn(0.4, u4));
      ch.st[2 * i] = u1;
      ch.st[2 * i + 1] = u3;
      ch.par[4 * i] = p1;
      ch.par[4 * i + 1] = __dsub_rn(0.5, p1);
      ch.par[4 * i + 2] = p2;
      ch.par[4 * i + 3] = __dsub_rn(0.5, p2);
    } else if (kind == 2) {  // logistic pair: x0 = u, r = 3.9 + 0.1 u
      const double u1 = unit_of(main_next_group(m));
      const double u2 = unit_of(main_next_group(m));
      const double u3 = unit_of(main_next_group(m));
      const double u4 = unit_of(main_next_group(m));
      ch.st[2 * i] = u1;
      ch.st[2 * i + 1] = u3;
      ch.par[4 * i] = __dadd_rn(3.9, __dmul_rn(0.1, u2));
      ch.par[4 * i + 1] = 0.0;
      ch.par[4 * i + 2] = __dadd_rn(3.9, __dmul_rn(0.1, u4));
      ch.par[4 * i + 3] = 0.0;
    } else {
      const double u1 = unit_of(main_next_group(m));
      const double u2 = unit_of(main_next_group(m));
      const double u3 = unit_of(main_next_group(m));
      const double u4 = unit_of(main_next_group(m));
      const double u5 = unit_of(main_next_group(m));
      const double u6 = unit_of(main_next_group(m));
      const double mu1 = __dadd_rn(0.44, __dmul_rn(0.49, u3));
      const double mu2 = __dadd_rn(0.44, __dmul_rn(0.49, u6));
      ch.st[4 * i] = u1;
      ch.st[4 * i + 1] = u2;
      ch.st[4 * i + 2] = u4;
      ch.st[4 * i + 3] = u5;
      ch.par[2 * i] = __dmul_rn(kPi, mu1);
      ch.par[2 * i + 1] = __dmul_rn(kPi, mu2);
    }
    ch.carry[2 * i] = 0;
    ch.carry[2 * i + 1] = 0;
    ch.carry_len[i] = 0;
  }
  *mp = m;
}

cudaError_t launch_key_schedule(int kind, MainPrbg* main, Chains ch, int n, cudaStream_t st) {
  k_key_schedule<<<1, 32, 0, st>>>(kind, main, ch, n);
  return cudaGetLastError();
}

// s_c of the next nframes frames (Alg. 1), serially from PRBG_m.
__device__ void frame_sc_serial(MainPrbg* mp, int nframes, long long* sc, int cap = 0, int slot0 = 0) {
  MainPrbg m = *mp;
  for (int f = 0; f < nframes; f++) sc[cap > 0 ? (slot0 + f) % cap : f] = 1 + (long long)(main_next_group(m) & 0xFFFFull);
  *mp = m;
}

__global__ void k_frame_sc(MainPrbg* mp, int nframes, long long* sc, int cap, int slot0) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  frame_sc_serial(mp, nframes, sc, cap, slot0);
}

// floor(s_c * csin((2 pi alpha) / H)) mod W, in [0, W).
__device__ __forceinline__ int kmod_of(const Layout& L, long long sc, int a) {
  const double t = __ddiv_rn(__dmul_rn(kTwoPi, (double)a), (double)L.H);
  const double v = __dmul_rn((double)sc, csin(t));
  long long k = (long long)floor(v) % L.W;
  if (k < 0) k += L.W;
  return (int)k;
}

// kmod[f][alpha] for the pass's frames (Eq. 1 shift table).
__global__ void k_kmod(Layout L, const long long* sc, int nframes, int* kmod, int cap, int slot0) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nframes * L.H) return;
  const int f = (int)(idx / L.H);
  const int a = (int)(idx - (long long)f * L.H);
  const int slot = cap > 0 ? (slot0 + f) % cap : f;
  kmod[(long long)slot * L.H + a] = kmod_of(L, sc[slot], a);
}

cudaError_t launch_frame_schedule(const Layout& L, MainPrbg* main, int nframes, long long* sc, int* kmod,
                                  cudaStream_t st, int cap, int slot0) {
  if (nframes <= 0) return cudaSuccess;
  k_frame_sc<<<1, 32, 0, st>>>(main, nframes, sc, cap, slot0);
  const long long tot = (long long)nframes * L.H;
  k_kmod<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(L, sc, nframes, kmod, cap, slot0);
  return cudaGetLastError();
}

// =============================================================================
// Keystream (Sec. 3): one thread per subframe chain, both maps of the pair in
// the same thread (two independent dependency chains).
// =============================================================================

// Writes a chain's byte stream into KS[f][j][q], q in [qstart, qend), round j
// after round j-1, merging bytes into aligned 8-byte words.  The first and
// last word of a range may be shared with the neighbouring subframe's chain:
// those are written byte by byte.
struct KsWriter {
  uint8_t* fbase;
  long long Npad;
  int rounds, j, q, qstart, qend;
  uint8_t* waddr;
  uint64_t acc;
  uint32_t mask;

  __device__ __forceinline__ void begin_round() {
    waddr = fbase + (long long)j * Npad + (q & ~7);
    acc = 0;
    mask = 0;
  }
  __device__ __forceinline__ void flush() {
    if (mask == 0xFFu) {
      *reinterpret_cast<uint64_t*>(waddr) = acc;
    } else if (mask) {
#pragma unroll
      for (int k = 0; k < 8; k++)
        if (mask & (1u << k)) waddr[k] = (uint8_t)(acc >> (8 * k));
    }
    acc = 0;
    mask = 0;
  }
  // Append the low `cnt` (1..8) bytes of v, lowest byte first.
  __device__ __forceinline__ void put(uint64_t v, int cnt) {
    while (cnt > 0) {
      const int room = qend - q;
      const int take = cnt < room ? cnt : room;
      const int s = q & 7;
      const int n1 = take < 8 - s ? take : 8 - s;
      const uint64_t m1 = (n1 == 8) ? ~0ull : ((1ull << (8 * n1)) - 1);
      acc |= (v & m1) << (8 * s);
      mask |= ((1u << n1) - 1u) << s;
      if (s + n1 == 8) {
        flush();
        waddr += 8;
      }
      if (take > n1) {  // remainder starts the next word (n1 < 8, n2 <= 7)
        const int n2 = take - n1;
        acc = (v >> (8 * n1)) & ((1ull << (8 * n2)) - 1);
        mask = (1u << n2) - 1u;
      }
      q += take;
      v = (take == 8) ? 0 : (v >> (8 * take));
      cnt -= take;
      if (q == qend) {
        flush();
        j++;
        q = qstart;
        if (j < rounds) begin_round();
      }
    }
  }
};

__device__ __forceinline__ void shr128(uint64_t& lo, uint64_t& hi, int bits) {
  if (bits == 0) return;
  if (bits >= 64) {
    lo = (bits >= 128) ? 0 : (hi >> (bits - 64));
    hi = 0;
  } else {
    lo = (lo >> bits) | (hi << (64 - bits));
    hi >>= bits;
  }
}

template <int KIND, bool INTDIV>
__global__ void __launch_bounds__(32) k_keystream(Layout L, Tables tb, Chains ch, int nframes, uint8_t* ks) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.n) return;
  constexpr int STEP = KIND == 1 ? 12 : 6;  // bytes per iterate of the pair (2DLASM: x and y)
  const int qstart = L.C * tb.pi[i];
  const int qend = L.C * tb.pi[i + 1];
  double x1, x2, y1 = 0, y2 = 0, p1 = 0, q1 = 0, p2 = 0, q2 = 0, pm1 = 0, pm2 = 0;
  if (KIND != 1) {  // PLCM: p, 1/2 - p per map; logistic: r, 0 per map
    x1 = ch.st[2 * i];
    x2 = ch.st[2 * i + 1];
    p1 = ch.par[4 * i];
    q1 = ch.par[4 * i + 1];
    p2 = ch.par[4 * i + 2];
    q2 = ch.par[4 * i + 3];
  } else {
    x1 = ch.st[4 * i];
    y1 = ch.st[4 * i + 1];
    x2 = ch.st[4 * i + 2];
    y2 = ch.st[4 * i + 3];
    pm1 = ch.par[2 * i];
    pm2 = ch.par[2 * i + 1];
  }
  PlcmMap m1{}, m2{};
  if (KIND == 0 && INTDIV) {
    m1 = make_plcm(p1, q1);
    m2 = make_plcm(p2, q2);
  }
  uint64_t c0 = ch.carry[2 * i], c1 = ch.carry[2 * i + 1];
  int clen = ch.carry_len[i];
  const long long per_frame = (long long)L.rounds * (qend - qstart);

  for (int f = 0; f < nframes; f++) {
    KsWriter w;
    w.fbase = ks + (long long)f * L.rounds * L.Npad;
    w.Npad = L.Npad;
    w.rounds = L.rounds;
    w.j = 0;
    w.q = qstart;
    w.qstart = qstart;
    w.qend = qend;
    w.begin_round();
    long long rem = per_frame;
    // 1. bytes left over from the previous frame's last iterate (R7)
    while (clen > 0 && rem > 0) {
      int take = clen < 8 ? clen : 8;
      if (take > rem) take = (int)rem;
      w.put(c0, take);
      shr128(c0, c1, 8 * take);
      clen -= take;
      rem -= take;
    }
    // 2. whole iterates
    while (rem >= STEP) {
      if (KIND == 2) {
        x1 = logistic_step(x1, p1);
        x2 = logistic_step(x2, p2);
        w.put(mant48(x1) ^ mant48(x2), 6);
      } else if (KIND == 0) {
        if (INTDIV) {
          x1 = plcm_step_int(x1, m1);
          x2 = plcm_step_int(x2, m2);
        } else {
          x1 = plcm_step(x1, p1, q1);
          x2 = plcm_step(x2, p2, q2);
        }
        w.put(mant48(x1) ^ mant48(x2), 6);
      } else {
        lasm_step(x1, y1, pm1);
        lasm_step(x2, y2, pm2);
        w.put(mant48(x1) ^ mant48(x2), 6);
        w.put(mant48(y1) ^ mant48(y2), 6);
      }
      rem -= STEP;
    }
    // 3. a last, partly used iterate; its other bytes carry over
    if (rem > 0) {
      uint64_t lo, hi;
      if (KIND == 2) {
        x1 = logistic_step(x1, p1);
        x2 = logistic_step(x2, p2);
        lo = mant48(x1) ^ mant48(x2);
        hi = 0;
      } else if (KIND == 0) {
        if (INTDIV) {
          x1 = plcm_step_int(x1, m1);
          x2 = plcm_step_int(x2, m2);
        } else {
          x1 = plcm_step(x1, p1, q1);
          x2 = plcm_step(x2, p2, q2);
        }
        lo = mant48(x1) ^ mant48(x2);
        hi = 0;
      } else {
        lasm_step(x1, y1, pm1);
        lasm_step(x2, y2, pm2);
        const uint64_t vx = mant48(x1) ^ mant48(x2), vy = mant48(y1) ^ mant48(y2);
        lo = vx | (vy << 48);
        hi = vy >> 16;
      }
      const int r = (int)rem;
      w.put(lo, r < 8 ? r : 8);
      if (r > 8) w.put(hi, r - 8);
      shr128(lo, hi, 8 * r);
      c0 = lo;
      c1 = hi;
      clen = STEP - r;
      rem = 0;
    }
  }
  if (KIND != 1) {
    ch.st[2 * i] = x1;
    ch.st[2 * i + 1] = x2;
  } else {
    ch.st[4 * i] = x1;
    ch.st[4 * i + 1] = y1;
    ch.st[4 * i + 2] = x2;
    ch.st[4 * i + 3] = y2;
  }
  ch.carry[2 * i] = c0;
  ch.carry[2 * i + 1] = c1;
  ch.carry_len[i] = clen;
}

// -----------------------------------------------------------------------------
// Keystream, lane-pair form: the two maps of subframe i run on lanes 2i and
// 2i+1 of a warp (one dependency chain per lane) and exchange their 6-byte
// groups with one shuffle.  Both lanes then hold the same byte stream and
// write it as aligned 8-byte words: 24 bytes (4 PLCM or 2 2DLASM iterates)
// advance the write position by 3 whole words, so the phase q mod 8 is the
// same at every group boundary and a group is three funnel shifts and three
// 8-byte stores.  Range heads and tails (shared words with the neighbouring
// subframes) go byte by byte.

__device__ __forceinline__ uint64_t fsh(uint64_t a, uint64_t b, int sh) {
  // (b:a) shifted left by sh bits, high word: b << sh | a >> (64 - sh); sh in [0, 56]
  return (b << sh) | ((a >> (63 - sh)) >> 1);
}

struct PairWriter {
  uint8_t* fb;     // keystream base of the current frame (round 0)
  long long Npad;
  int j, q, qs, qe, side;
  uint64_t acc;    // bytes [0, q mod 8) of the word containing q
  uint32_t own;    // which of them belong to this subframe's range

  __device__ __forceinline__ uint8_t* word_ptr(int qq) const { return fb + (long long)j * Npad + (qq & ~7); }
  __device__ __forceinline__ void flush(int qq) {
    if (side == 0 && own) {
      uint8_t* a = word_ptr(qq);
      if (own == 0xFFu) {
        *reinterpret_cast<uint64_t*>(a) = acc;
      } else {
#pragma unroll
        for (int k = 0; k < 8; k++)
          if (own & (1u << k)) a[k] = (uint8_t)(acc >> (8 * k));
      }
    }
    acc = 0;
    own = 0;
  }
  __device__ __forceinline__ void end_of_range_check() {
    if (q == qe) {
      flush(q - 1);
      j++;
      q = qs;
    }
  }
  // Append the low cnt (0..8) bytes of v, one at a time.
  __device__ __forceinline__ void put_slow(uint64_t v, int cnt) {
    for (int k = 0; k < cnt; k++) {
      const int ph = q & 7;
      acc |= ((v >> (8 * k)) & 0xFFull) << (8 * ph);
      own |= 1u << ph;
      q++;
      if (q == qe) {
        flush(q - 1);
        j++;
        q = qs;
      } else if ((q & 7) == 0) {
        flush(q - 1);
      }
    }
  }
  __device__ __forceinline__ bool fast_ok() const { return q + 24 <= qe && own == ((1u << (q & 7)) - 1u); }
  // Append 24 bytes without the end-of-range test (the caller knows q + 24 < qe
  // or tests afterwards).
  __device__ __forceinline__ void put24_raw(uint64_t c0, uint64_t c1, uint64_t c2) {
    const int sh = 8 * (q & 7);
    const uint64_t w0 = acc | (c0 << sh);
    const uint64_t w1 = fsh(c0, c1, sh);
    const uint64_t w2 = fsh(c1, c2, sh);
    acc = (c2 >> (63 - sh)) >> 1;
    uint64_t* a = reinterpret_cast<uint64_t*>(word_ptr(q));
    // even lane: words 0 and 2; odd lane: word 1 (one predicated second store)
    a[side] = side ? w1 : w0;
    if (side == 0) a[2] = w2;
    q += 24;
  }
  // put24_raw at a word boundary with nothing pending (q mod 8 = 0, own = 0).
  __device__ __forceinline__ void put24_aligned(uint64_t c0, uint64_t c1, uint64_t c2) {
    uint64_t* a = reinterpret_cast<uint64_t*>(word_ptr(q));
    a[side] = side ? c1 : c0;
    if (side == 0) a[2] = c2;
    q += 24;
  }
  // Append 24 bytes c0 | c1 | c2 (little-endian order).
  __device__ __forceinline__ void put24(uint64_t c0, uint64_t c1, uint64_t c2) {
    const int sh = 8 * (q & 7);
    const uint64_t w0 = acc | (c0 << sh);
    const uint64_t w1 = fsh(c0, c1, sh);
    const uint64_t w2 = fsh(c1, c2, sh);
    acc = (c2 >> (63 - sh)) >> 1;
    uint64_t* a = reinterpret_cast<uint64_t*>(word_ptr(q));
    if (side == 0) {
      a[0] = w0;
      a[2] = w2;
    } else {
      a[1] = w1;
    }
    q += 24;
    end_of_range_check();
  }
};

// Keystream base of frame f of a call: frames laid end to end (cap = 0), or a
// ring of cap frame slots starting at slot0 (the batches' run-ahead rings).
__device__ __forceinline__ uint8_t* ks_frame(uint8_t* ks, const Layout& L, int f, int cap, int slot0) {
  const int slot = cap > 0 ? (slot0 + f) % cap : f;
  return ks + (long long)slot * L.rounds * L.Npad;
}

// SINE_B64: the 2DLASM sines with the all-binary64 reduction (shorter chain,
// for kernels that hold whole SMs); otherwise the integer-assisted reduction
// (fewer binary64 operations, for chains that share the SMs).
template <int KIND, bool FX, bool SINE_B64 = false>
__device__ __forceinline__ void ks_pair_chain(const Layout& L, const Tables& tb, const Chains& ch, int nframes,
                                              uint8_t* ks, const int i, const int side, int cap = 0, int slot0 = 0) {
  if (i >= L.n) return;  // both lanes of a pair leave together
  const unsigned pmask = 3u << (threadIdx.x & 30);
  constexpr int STEP = KIND == 1 ? 12 : 6;  // 2DLASM: x and y per iterate

  double x = 0, y = 0, p = 0, qd = 0, pm = 0;
  uint64_t xb = 0;
  PlcmFx F{};
  bool fx_ok = false;
  if (KIND != 1) {  // PLCM (p, 1/2 - p) or logistic (r, 0) per map
    x = ch.st[2 * i + side];
    p = ch.par[4 * i + 2 * side];
    qd = ch.par[4 * i + 2 * side + 1];
    xb = (uint64_t)__double_as_longlong(x);
    if (FX && KIND == 0) fx_ok = make_plcm_fx(p, qd, F);
  } else {
    x = ch.st[4 * i + 2 * side];
    y = ch.st[4 * i + 2 * side + 1];
    pm = ch.par[2 * i + side];
  }
  uint64_t c0 = ch.carry[2 * i], c1 = ch.carry[2 * i + 1];
  int clen = ch.carry_len[i];

  PairWriter w;
  w.Npad = L.Npad;
  w.qs = L.C * tb.pi[i];
  w.qe = L.C * tb.pi[i + 1];
  w.side = side;
  const long long per_frame = (long long)L.rounds * (w.qe - w.qs);

  // one PLCM iterate of this lane's map; the pair's XORed 6-byte group
  auto plcm_next = [&]() -> uint64_t {
    if (KIND == 2) {
      xb = (uint64_t)__double_as_longlong(logistic_step(__longlong_as_double((long long)xb), p));
    } else if (FX) {
      bool ok = true;
      uint64_t nb = fx_ok ? plcm_fx_step(xb, F, ok) : 0;
      if (!fx_ok || !ok) nb = (uint64_t)__double_as_longlong(plcm_step(__longlong_as_double((long long)xb), p, qd));
      xb = nb;
    } else {
      xb = (uint64_t)__double_as_longlong(plcm_step(__longlong_as_double((long long)xb), p, qd));
    }
    const uint64_t own48 = xb & 0xFFFFFFFFFFFFull;
    return own48 ^ __shfl_xor_sync(pmask, own48, 1);
  };
  auto lasm_next = [&](uint64_t& vx, uint64_t& vy) {
    lasm_step<SINE_B64>(x, y, pm);
    const uint64_t ox = mant48(x), oy = mant48(y);
    vx = ox ^ __shfl_xor_sync(pmask, ox, 1);
    vy = oy ^ __shfl_xor_sync(pmask, oy, 1);
  };

  for (int f = 0; f < nframes; f++) {
    w.fb = ks_frame(ks, L, f, cap, slot0);
    w.j = 0;
    w.q = w.qs;
    w.acc = 0;
    w.own = 0;
    long long rem = per_frame;
    while (clen > 0 && rem > 0) {  // bytes left over from the last iterate (R7)
      int take = clen < 8 ? clen : 8;
      if (take > rem) take = (int)rem;
      w.put_slow(c0, take);
      shr128(c0, c1, 8 * take);
      clen -= take;
      rem -= take;
    }
    while (rem > 0) {
      if (rem >= 24 && w.fast_ok()) {
        uint64_t a0, a1, a2, a3;
        if (KIND != 1) {
          a0 = plcm_next();
          a1 = plcm_next();
          a2 = plcm_next();
          a3 = plcm_next();
        } else {
          lasm_next(a0, a1);
          lasm_next(a2, a3);
        }
        w.put24(a0 | (a1 << 48), (a1 >> 16) | (a2 << 32), (a2 >> 32) | (a3 << 16));
        rem -= 24;
      } else {
        uint64_t lo, hi = 0;
        if (KIND != 1) {
          lo = plcm_next();
        } else {
          uint64_t vx, vy;
          lasm_next(vx, vy);
          lo = vx | (vy << 48);
          hi = vy >> 16;
        }
        const int take = rem < STEP ? (int)rem : STEP;
        w.put_slow(lo, take < 8 ? take : 8);
        if (take > 8) w.put_slow(hi, take - 8);
        if (take < STEP) {  // keep the rest of the iterate for the next frame
          shr128(lo, hi, 8 * take);
          c0 = lo;
          c1 = hi;
          clen = STEP - take;
        }
        rem -= take;
      }
    }
  }
  if (KIND != 1) {
    ch.st[2 * i + side] = __longlong_as_double((long long)xb);
  } else {
    ch.st[4 * i + 2 * side] = x;
    ch.st[4 * i + 2 * side + 1] = y;
  }
  if (side == 0) {
    ch.carry[2 * i] = c0;
    ch.carry[2 * i + 1] = c1;
    ch.carry_len[i] = clen;
  }
}

template <int KIND, bool FX>
__global__ void __launch_bounds__(32) k_ks_pair(Layout L, Tables tb, Chains ch, int nframes, uint8_t* ks, int cap,
                                                int slot0) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  ks_pair_chain<KIND, FX>(L, tb, ch, nframes, ks, gt >> 1, gt & 1, cap, slot0);
}

// PLCM keystream on the integer pipes, lane-pair form with the writes of a
// 24-byte group overlapped with the iterates of the next group: in the steady
// loop a lane issues two iterates, stores the previous group (whose partner
// bytes were exchanged a whole group earlier, so the shuffle latency is
// hidden), then two more iterates.  The fallback for operands outside the
// fixed-point range is checked once per group: the rare group that needs it
// is recomputed step by step with the hardware division.
__device__ __forceinline__ void ks_plcm_fx_chain(const Layout& L, const Tables& tb, const Chains& ch, int nframes,
                                                 uint8_t* ks, const int i, const int side, int cap = 0,
                                                 int slot0 = 0, int force_fallback = 0) {
  if (i >= L.n) return;
  const unsigned pmask = 3u << (threadIdx.x & 30);
  constexpr uint64_t M48 = 0xFFFFFFFFFFFFull;

  const double p = ch.par[4 * i + 2 * side];
  const double qd = ch.par[4 * i + 2 * side + 1];
  uint64_t xb = (uint64_t)__double_as_longlong(ch.st[2 * i + side]);
  PlcmFx F;
  // force_fallback (a test mode): 1 = every fixed-point iterate counts as out
  // of range, so each range is computed and then rewritten by the exact
  // fallback; 2 = the same for odd subframes only (pairs of one warp diverge)
  const bool forced = force_fallback == 1 || (force_fallback == 2 && (i & 1));
  const bool fx_ok = make_plcm_fx(p, qd, F) && !forced;
  uint64_t c0 = ch.carry[2 * i], c1 = ch.carry[2 * i + 1];
  int clen = ch.carry_len[i];

  PairWriter w;
  w.Npad = L.Npad;
  w.qs = L.C * tb.pi[i];
  w.qe = L.C * tb.pi[i + 1];
  w.side = side;
  const long long per_frame = (long long)L.rounds * (w.qe - w.qs);

  auto safe_step = [&](uint64_t b) -> uint64_t {
    bool ok = false;
    uint64_t r = fx_ok ? plcm_fx_step(b, F, ok) : 0;
    if (!ok) r = (uint64_t)__double_as_longlong(plcm_step(__longlong_as_double((long long)b), p, qd));
    return r;
  };
  // own map's 24 bytes of 4 iterates as 3 words; the fix-up path recomputes
  auto fix_group = [&](uint64_t x0, uint64_t& a, uint64_t& b, uint64_t& c, uint64_t& d) {
    a = safe_step(x0);
    b = safe_step(a);
    c = safe_step(b);
    d = safe_step(c);
  };
  auto pack = [&](uint64_t a, uint64_t b, uint64_t c, uint64_t d, uint64_t& o0, uint64_t& o1, uint64_t& o2) {
    a &= M48;
    b &= M48;
    c &= M48;
    d &= M48;
    o0 = a | (b << 48);
    o1 = (b >> 16) | (c << 32);
    o2 = (c >> 32) | (d << 16);
  };

  for (int f = 0; f < nframes; f++) {
    w.fb = ks_frame(ks, L, f, cap, slot0);
    w.j = 0;
    w.q = w.qs;
    w.acc = 0;
    w.own = 0;
    long long rem = per_frame;
    while (clen > 0 && rem > 0) {  // bytes left over from the last iterate (R7)
      int take = clen < 8 ? clen : 8;
      if (take > rem) take = (int)rem;
      w.put_slow(c0, take);
      shr128(c0, c1, 8 * take);
      clen -= take;
      rem -= take;
    }
    // G groups of 24 bytes; ALIGNED: the range position is a word boundary,
    // so the group's three words need no funnel shifts.  FULL: every lane of
    // the warp runs this same loop the same number of times, so the partner
    // exchange can name the whole warp (a shuffle restricted to the lane pair
    // costs about 60 cycles more per iterate).  The loop body is one basic
    // block: iteration g computes group g, packs and exchanges group g - 1 and
    // stores group g - 2; the fixed-point range flags are accumulated, and a
    // pair with an iterate outside it (about 2^-30 per iterate) redoes the
    // range step by step with the exact fallback.
    auto run_groups = [&](long long G, auto aligned, auto full) {
      const unsigned mk = decltype(full)::value ? 0xFFFFFFFFu : pmask;
      auto put = [&](uint64_t c0, uint64_t c1, uint64_t c2) {
        if (decltype(aligned)::value)
          w.put24_aligned(c0, c1, c2);
        else
          w.put24_raw(c0, c1, c2);
      };
      const uint64_t x_start = xb;
      const int q_start = w.q, j_start = w.j;
      const uint64_t acc_start = w.acc;
      const uint32_t own_start = w.own;
      bool good = fx_ok;
      uint64_t ra, rb, rc, rd;              // iterates of the previous group
      uint64_t o0 = 0, o1 = 0, o2 = 0, s0 = 0, s1 = 0, s2 = 0;  // own and partner words of the one before
      {
        bool k0, k1, k2, k3;
        ra = plcm_fx_step(xb, F, k0);
        rb = plcm_fx_step(ra, F, k1);
        rc = plcm_fx_step(rb, F, k2);
        rd = plcm_fx_step(rc, F, k3);
        good &= k0 & k1 & k2 & k3;
        xb = rd;
      }
      if (G >= 2) {
        bool k0, k1, k2, k3;
        const uint64_t a = plcm_fx_step(xb, F, k0);
        const uint64_t b = plcm_fx_step(a, F, k1);
        pack(ra, rb, rc, rd, o0, o1, o2);
        s0 = __shfl_xor_sync(mk, o0, 1);
        s1 = __shfl_xor_sync(mk, o1, 1);
        s2 = __shfl_xor_sync(mk, o2, 1);
        const uint64_t c = plcm_fx_step(b, F, k2);
        const uint64_t d = plcm_fx_step(c, F, k3);
        good &= k0 & k1 & k2 & k3;
        xb = d;
        ra = a;
        rb = b;
        rc = c;
        rd = d;
      }
      for (int g = 2; g < (int)G; g++) {
        bool k0, k1, k2, k3;
        const uint64_t a = plcm_fx_step(xb, F, k0);
        const uint64_t b = plcm_fx_step(a, F, k1);
        put(o0 ^ s0, o1 ^ s1, o2 ^ s2);  // group g - 2
        pack(ra, rb, rc, rd, o0, o1, o2);  // group g - 1
        s0 = __shfl_xor_sync(mk, o0, 1);
        s1 = __shfl_xor_sync(mk, o1, 1);
        s2 = __shfl_xor_sync(mk, o2, 1);
        const uint64_t c = plcm_fx_step(b, F, k2);
        const uint64_t d = plcm_fx_step(c, F, k3);
        good &= k0 & k1 & k2 & k3;
        xb = d;
        ra = a;
        rb = b;
        rc = c;
        rd = d;
      }
      if (G >= 2) put(o0 ^ s0, o1 ^ s1, o2 ^ s2);
      pack(ra, rb, rc, rd, o0, o1, o2);
      s0 = __shfl_xor_sync(mk, o0, 1);
      s1 = __shfl_xor_sync(mk, o1, 1);
      s2 = __shfl_xor_sync(mk, o2, 1);
      put(o0 ^ s0, o1 ^ s1, o2 ^ s2);
      // every lane of mk takes part in the exchange (no short circuit)
      const int partner_good = __shfl_xor_sync(mk, good ? 1 : 0, 1);
      const bool pair_good = good && partner_good != 0;
      if (!pair_good) {  // both lanes of the pair: rewrite the range exactly
        xb = x_start;
        w.q = q_start;
        w.j = j_start;
        w.acc = acc_start;
        w.own = own_start;
        for (long long g = 0; g < G; g++) {
          uint64_t a, b, c, d;
          fix_group(xb, a, b, c, d);
          xb = d;
          pack(a, b, c, d, o0, o1, o2);
          s0 = __shfl_xor_sync(pmask, o0, 1);
          s1 = __shfl_xor_sync(pmask, o1, 1);
          s2 = __shfl_xor_sync(pmask, o2, 1);
          put(o0 ^ s0, o1 ^ s1, o2 ^ s2);
        }
      }
    };
    while (rem > 0) {
      if (rem >= 24 && w.fast_ok()) {
        long long G = (w.qe - w.q) / 24;
        if (G > rem / 24) G = rem / 24;
        const bool aligned = (w.q & 7) == 0;
        // warp-uniform loop: all 32 lanes here together with the same count and phase
        const unsigned key = (unsigned)G * 2u + (aligned ? 1u : 0u);
        bool uniform = false;
        if (__activemask() == 0xFFFFFFFFu)
          uniform = __reduce_min_sync(0xFFFFFFFFu, key) == __reduce_max_sync(0xFFFFFFFFu, key);
        if (uniform) {
          if (aligned)
            run_groups(G, std::true_type{}, std::true_type{});
          else
            run_groups(G, std::false_type{}, std::true_type{});
        } else if (aligned) {
          run_groups(G, std::true_type{}, std::false_type{});
        } else {
          run_groups(G, std::false_type{}, std::false_type{});
        }
        w.end_of_range_check();
        rem -= 24 * G;
      } else {
        const uint64_t nb = safe_step(xb);
        xb = nb;
        const uint64_t own48 = nb & M48;
        const uint64_t v = own48 ^ __shfl_xor_sync(pmask, own48, 1);
        const int take = rem < 6 ? (int)rem : 6;
        w.put_slow(v, take);
        if (take < 6) {  // keep the rest of the iterate for the next frame
          c0 = v >> (8 * take);
          c1 = 0;
          clen = 6 - take;
        }
        rem -= take;
      }
    }
  }
  ch.st[2 * i + side] = __longlong_as_double((long long)xb);
  if (side == 0) {
    ch.carry[2 * i] = c0;
    ch.carry[2 * i + 1] = c1;
    ch.carry_len[i] = clen;
  }
}

__global__ void __launch_bounds__(32) k_ks_plcm_fx(Layout L, Tables tb, Chains ch, int nframes, uint8_t* ks, int cap,
                                                   int slot0, int force_fallback) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  ks_plcm_fx_chain(L, tb, ch, nframes, ks, gt >> 1, gt & 1, cap, slot0, force_fallback);
}

// The same chains in CTAs of up to 4 warps (one per SM sub-partition)
// launched with the SM's whole shared memory (unused): one CTA per SM, and no
// other kernel's CTA that needs shared memory can join it.  (A bound of 256
// threads makes the compiler schedule the chain about 15% slower; 128 threads
// with one CTA per SM about 3% faster than 128 alone.)
__global__ void __launch_bounds__(128, 1) k_ks_plcm_fx_sm(Layout L, Tables tb, Chains ch, int nframes, uint8_t* ks,
                                                       int cap, int slot0, int force_fallback) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  ks_plcm_fx_chain(L, tb, ch, nframes, ks, gt >> 1, gt & 1, cap, slot0, force_fallback);
}

template <int KIND>
__global__ void __launch_bounds__(128) k_ks_pair_sm(Layout L, Tables tb, Chains ch, int nframes, uint8_t* ks, int cap,
                                                    int slot0) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  ks_pair_chain<KIND, false, true>(L, tb, ch, nframes, ks, gt >> 1, gt & 1, cap, slot0);
}

static int reserve_smem_bytes() {
  static int bytes[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 0;
  if (bytes[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 48 * 1024;
    bytes[dev] = v;
  }
  return bytes[dev];
}

cudaError_t launch_keystream(int kind, const Layout& L, Tables tb, Chains ch, int nframes, uint8_t* ks,
                             int plcm_int, cudaStream_t st, int cap, int slot0, int sm_warps) {
  if (nframes <= 0) return cudaSuccess;
  if (sm_warps > 0) {
    const int threads = 32 * (sm_warps > 4 ? 4 : sm_warps);
    const int blocks = (2 * L.n + threads - 1) / threads;
    const int smem = reserve_smem_bytes();
    cudaError_t e;
    if (kind == 0 && plcm_int) {
      e = allow_smem(k_ks_plcm_fx_sm, smem);
      if (e != cudaSuccess) return e;
      k_ks_plcm_fx_sm<<<blocks, threads, smem, st>>>(L, tb, ch, nframes, ks, cap, slot0,
                                                     plcm_int >= 2 ? plcm_int - 1 : 0);
    } else if (kind == 0) {
      e = allow_smem(k_ks_pair_sm<0>, smem);
      if (e != cudaSuccess) return e;
      k_ks_pair_sm<0><<<blocks, threads, smem, st>>>(L, tb, ch, nframes, ks, cap, slot0);
    } else if (kind == 2) {
      e = allow_smem(k_ks_pair_sm<2>, smem);
      if (e != cudaSuccess) return e;
      k_ks_pair_sm<2><<<blocks, threads, smem, st>>>(L, tb, ch, nframes, ks, cap, slot0);
    } else {
      e = allow_smem(k_ks_pair_sm<1>, smem);
      if (e != cudaSuccess) return e;
      k_ks_pair_sm<1><<<blocks, threads, smem, st>>>(L, tb, ch, nframes, ks, cap, slot0);
    }
    return cudaGetLastError();
  }
  const int blocks = (2 * L.n + 31) / 32;
  if (kind == 0 && plcm_int)
    k_ks_plcm_fx<<<blocks, 32, 0, st>>>(L, tb, ch, nframes, ks, cap, slot0, plcm_int >= 2 ? plcm_int - 1 : 0);
  else if (kind == 0)
    k_ks_pair<0, false><<<blocks, 32, 0, st>>>(L, tb, ch, nframes, ks, cap, slot0);
  else if (kind == 2)
    k_ks_pair<2, false><<<blocks, 32, 0, st>>>(L, tb, ch, nframes, ks, cap, slot0);
  else
    k_ks_pair<1, false><<<blocks, 32, 0, st>>>(L, tb, ch, nframes, ks, cap, slot0);
  return cudaGetLastError();
}

// The earlier one-thread-per-subframe form (both maps in one thread), kept for
// comparison measurements.
cudaError_t launch_keystream_thread(int kind, const Layout& L, Tables tb, Chains ch, int nframes, uint8_t* ks,
                                    int plcm_int, cudaStream_t st) {
  if (nframes <= 0) return cudaSuccess;
  const int blocks = (L.n + 31) / 32;
  if (kind == 0 && plcm_int)
    k_keystream<0, true><<<blocks, 32, 0, st>>>(L, tb, ch, nframes, ks);
  else if (kind == 0)
    k_keystream<0, false><<<blocks, 32, 0, st>>>(L, tb, ch, nframes, ks);
  else if (kind == 2)
    k_keystream<2, false><<<blocks, 32, 0, st>>>(L, tb, ch, nframes, ks);
  else
    k_keystream<1, false><<<blocks, 32, 0, st>>>(L, tb, ch, nframes, ks);
  return cudaGetLastError();
}

// =============================================================================
// Rounds
// =============================================================================
//
// Encryption round (Eq. 1 then Eq. 3), one CTA per (row-band tile of the
// OUTPUT frame, frame).  Output rows alpha in [a0, a0+T) of the confused frame
// Y need Z[alpha][o] = X[(alpha - o) mod H][o] (the column shear) followed by
// the row rotation Y[alpha][beta] = Z[alpha][(beta - k(alpha)) mod W].  Source
// row a contributes the contiguous columns o = (alpha - a) mod H (+ m H), one
// per output row, so the gather reads T consecutive pixels per source row into
// shared memory (one 32-bit slot per pixel for C = 3 and 4, see
// tile_row_stride).  The tile's bytes are then diffused in raster order as a
// segmented XOR scan: c_q = c_{q-1} xor d_q with d_q = b xor (y_q + b), reset to
// s_d xor d_q at every subframe start (Eq. 3 with the seed of Alg. 2).
//
// Each warp diffuses one sub-tile (R rows) on its own: 16 bytes per lane, a
// warp-shuffle scan per 512 bytes and a running carry, with no barrier.  The
// bytes of a sub-tile before its first subframe start are left relative to its
// first byte: bytes q < fixlim[s] hold c_q xor c(end of sub-tile s-1).  The
// value at the sub-tile's last byte is written to agg_out; the next round (or
// k_enc_fixup after the last round) scans these per-sub-tile values and applies
// the missing prefix while reading.  No CTA or warp waits on another.

// Segmented-scan element: bit 8 = "a subframe start lies in the span",
// bits 0..7 = XOR value (relative to the span's start if no start).
__device__ __forceinline__ uint32_t seg_combine(uint32_t a, uint32_t b) {
  return (b & 0x100u) ? b : ((a & 0x100u) | ((a ^ b) & 0xFFu));
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x = seg_combine(o, x);
  }
  return x;
}

// Carries of the two diffusion readings: a byte per chain for R4 (one chain
// over the subframe's bytes), a pixel word for R4' (one chain per channel,
// the C bytes of a pixel side by side).  A scan element holds the XOR value
// and, above it, the flag "a subframe start lies in the span".
template <bool PC>
struct CarryT {
  using V = uint32_t;  // scan element: bit 8 flag, bits 0..7 value
  using E = uint8_t;   // stored carry / aggregate
  static constexpr V F = 0x100u, M = 0xFFu;
};
template <>
struct CarryT<true> {
  using V = uint64_t;  // bit 32 flag, bits 0..31 value
  using E = uint32_t;
  static constexpr V F = 1ull << 32, M = 0xFFFFFFFFull;
};

template <bool PC>
__device__ __forceinline__ typename CarryT<PC>::V seg_comb(typename CarryT<PC>::V a, typename CarryT<PC>::V b) {
  using T = CarryT<PC>;
  return (b & T::F) ? b : ((a & T::F) | ((a ^ b) & T::M));
}

template <bool PC>
__device__ __forceinline__ typename CarryT<PC>::V warp_scan_t(typename CarryT<PC>::V x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const typename CarryT<PC>::V o = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x = seg_comb<PC>(o, x);
  }
  return x;
}

// s_carry[s] = true ciphertext value (R4: byte, R4': pixel word) at the end of
// sub-tile s-1, for all NS sub-tiles of the frame, by every warp of the block:
// warp w scans its share [s0, s1) of the aggregates relative to the share's
// start, the shares' totals (s_tot, one element per warp) then give each share
// its incoming value, which the entries before the share's first subframe
// start still miss.  Ends with a barrier; every thread of the block must call
// it.
__device__ __forceinline__ bool sub_flag(const Layout& L, const Tables& tb, int s, int rowb) {
  return __ldg(&tb.fixlim[s]) < min(L.H, (s + 1) * L.R) * rowb;  // a subframe starts in sub-tile s
}

template <bool PC>
__device__ void sub_carries_t(const Layout& L, const Tables& tb, const typename CarryT<PC>::E* agg,
                              typename CarryT<PC>::E* s_carry, typename CarryT<PC>::V* s_tot) {
  using T = CarryT<PC>;
  using V = typename T::V;
  using E = typename T::E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rowb = L.W * L.C;
  const int share = (((L.NS + nw - 1) / nw) + 31) & ~31;
  const int s0 = min(L.NS, warp * share), s1 = min(L.NS, s0 + share);
  V run = 0;
  for (int base = s0; base < s1; base += 32) {
    const int s = base + lane;
    V x = 0;
    if (s < s1) x = (sub_flag(L, tb, s, rowb) ? T::F : (V)0) | (V)agg[s];
    x = seg_comb<PC>(run, warp_scan_t<PC>(x));
    if (s < s1 && s + 1 < L.NS) s_carry[s + 1] = (E)x;
    run = __shfl_sync(0xFFFFFFFFu, x, 31);
  }
  if (lane == 0) s_tot[warp] = run;
  __syncthreads();
  V in = 0;  // value at the end of sub-tile s0 - 1
  for (int k = 0; k < warp; k++) in = seg_comb<PC>(in, s_tot[k]);
  if ((in & T::M) != 0) {
    for (int base = s0; base < s1; base += 32) {
      const int s = base + lane;
      const bool flag = s < s1 && sub_flag(L, tb, s, rowb);
      const uint32_t fl = __ballot_sync(0xFFFFFFFFu, flag);
      // entries whose share holds no start at or before them are relative
      const bool rel = s < s1 && (fl & (0xFFFFFFFFu >> (31 - lane))) == 0;
      if (rel && s + 1 < L.NS) s_carry[s + 1] ^= (E)(in & T::M);
      if (fl != 0) break;  // every later entry of the share is absolute
    }
  }
  if (threadIdx.x == 0) s_carry[0] = 0;
  __syncthreads();
}

__device__ __forceinline__ void sub_carries(const Layout& L, const Tables& tb, const uint8_t* agg, uint8_t* s_carry,
                                            uint32_t* s_tot) {
  sub_carries_t<false>(L, tb, agg, s_carry, s_tot);
}

__device__ __forceinline__ int mod_h(int v, int H) {
  v %= H;
  return v < 0 ? v + H : v;
}

// Subframe starts at pixels < p: #{i : floor(i P / n) < p} = min(n, ceil(p n / P)).
__device__ __forceinline__ int starts_before(const Layout& L, int p) {
  const long long r = ((long long)p * L.n + L.P - 1) / L.P;
  return r < L.n ? (int)r : L.n;
}

// Bytes j of the word holding chunk bytes w0 .. w0 + 3 with w0 + j >= k.
__device__ __forceinline__ uint32_t mask_from(int k, int w0) {
  const int kk = k - w0;
  return kk <= 0 ? 0xFFFFFFFFu : (kk >= 4 ? 0u : (0xFFFFFFFFu << (8 * kk)));
}

// Byte-wise a + b mod 256 in each of the four bytes of a word.
__device__ __forceinline__ uint32_t vadd4(uint32_t a, uint32_t b) {
  return ((a & 0x7F7F7F7Fu) + (b & 0x7F7F7F7Fu)) ^ ((a ^ b) & 0x80808080u);
}
// Byte-wise a - b mod 256 in each of the four bytes of a word.
__device__ __forceinline__ uint32_t vsub4(uint32_t a, uint32_t b) {
  return ((a | 0x80808080u) - (b & 0x7F7F7F7Fu)) ^ ((a ^ ~b) & 0x80808080u);
}
// Byte 3 of w in all four bytes.
__device__ __forceinline__ uint32_t bcast3(uint32_t w) { return __byte_perm(w, 0u, 0x3333u); }

// A byte repeated over the C bytes of a pixel word.
template <int C>
__device__ __forceinline__ uint32_t rep_px(uint32_t b) {
  return C == 1 ? b : (C == 3 ? b * 0x010101u : b * 0x01010101u);
}

// Shared-memory slot of pixel (tile row tt, column o): a word index for C = 3
// and 4 (one word per pixel, a skipped word after every 32), a byte index for
// C = 1.
template <int C>
__device__ __forceinline__ int zslot(const Layout& L, int tt, int o) {
  return C == 1 ? tt * L.ZS + o : tt * L.ZS + o + (o >> 5);
}

template <int C>
__device__ __forceinline__ void store_z(uint8_t* Z, int slot, uint32_t v) {
  if (C == 1)
    Z[slot] = (uint8_t)v;
  else
    reinterpret_cast<uint32_t*>(Z)[slot] = v;
}

// Byte ch of pixel (tt, o) of the tile in shared memory.
template <int C>
__device__ __forceinline__ uint8_t z_byte(const Layout& L, const uint8_t* Z, int tt, int o, int ch) {
  return C == 1 ? Z[zslot<1>(L, tt, o)] : Z[4 * zslot<C>(L, tt, o) + ch];
}

// The C bytes of the pixel at byte qx of frame X as the low bytes of a word
// (the rest zero).  aligned: X is 4-byte aligned, so the aligned words that
// hold the pixel lie in the frame whenever qx + 8 <= N; otherwise byte loads.
template <int C>
__device__ __forceinline__ uint32_t load_px_g(const uint8_t* X, int qx, bool aligned, int N) {
  if (C == 4 && aligned) return __ldg(reinterpret_cast<const uint32_t*>(X + qx));
  if (C == 3 && aligned && qx + 8 <= N) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(X + (qx & ~3));
    const uint32_t w0 = __ldg(w);
    const uint32_t w1 = (qx & 3) >= 2 ? __ldg(w + 1) : 0u;
    return __funnelshift_r(w0, w1, (uint32_t)(qx & 3) * 8u) & 0xFFFFFFu;
  }
  uint32_t v = 0;
#pragma unroll
  for (int c = 0; c < C; c++) v |= (uint32_t)__ldg(X + qx + c) << (8 * c);
  return v;
}

// Packed bytes zs .. zs + 15 of tile row tt (columns taken cyclically mod W,
// as the row rotation of Eq. 1 reads them) as four words, byte 0 lowest.
// C = 1 needs zs + 16 <= W or W a multiple of 4 (the caller checks).
template <int C>
__device__ __forceinline__ void z_row16(const Layout& L, const uint8_t* Z, int tt, int zs, uint32_t& y0,
                                        uint32_t& y1, uint32_t& y2, uint32_t& y3) {
  const uint32_t* Zw = reinterpret_cast<const uint32_t*>(Z);
  if (C == 4) {  // zs is a multiple of 4: four whole pixels
    uint32_t w[4];
    const int p = zs >> 2;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      int q = p + i;
      if (q >= L.W) q -= L.W;
      w[i] = Zw[zslot<4>(L, tt, q)];
    }
    y0 = w[0];
    y1 = w[1];
    y2 = w[2];
    y3 = w[3];
  } else if (C == 3) {  // six pixels cover bytes zs .. zs + 15 (zs = 3 p + ph)
    const int p = zs / 3, ph = zs - 3 * p;
    uint32_t w[6];
    const int base = tt * L.ZS;
    if (p + 5 < L.W) {
      const int s0 = base + p + (p >> 5), lo = p & 31;
#pragma unroll
      for (int i = 0; i < 6; i++) w[i] = Zw[s0 + i + ((lo + i) >> 5)];
    } else {
#pragma unroll
      for (int i = 0; i < 6; i++) {
        int q = p + i;
        if (q >= L.W) q -= L.W;
        w[i] = Zw[base + q + (q >> 5)];
      }
    }
    // the six 3-byte pixels as 18 consecutive bytes (k4 holds bytes 16, 17)
    const uint32_t k0 = __byte_perm(w[0], w[1], 0x4210u);
    const uint32_t k1 = __byte_perm(w[1], w[2], 0x5421u);
    const uint32_t k2 = __byte_perm(w[2], w[3], 0x6542u);
    const uint32_t k3 = __byte_perm(w[4], w[5], 0x4210u);
    const uint32_t k4 = __byte_perm(w[5], 0u, 0x4421u);
    const uint32_t sh = 8u * (uint32_t)ph;
    y0 = __funnelshift_r(k0, k1, sh);
    y1 = __funnelshift_r(k1, k2, sh);
    y2 = __funnelshift_r(k2, k3, sh);
    y3 = __funnelshift_r(k3, k4, sh);
  } else {  // bytes; the five words wrap word-wise at the row end when W is whole words
    uint32_t z0, z1, z2, z3, z4, sh;
    if (zs + 16 <= L.W) {
      const int za = tt * L.ZS + zs;
      const uint32_t* zw = reinterpret_cast<const uint32_t*>(Z + (za & ~3));
      sh = (uint32_t)(za & 3) * 8u;
      z0 = zw[0];
      z1 = zw[1];
      z2 = zw[2];
      z3 = zw[3];
      z4 = zw[4];
    } else {
      const uint32_t* zr = reinterpret_cast<const uint32_t*>(Z + tt * L.ZS);
      const int rw = L.W >> 2, wi = zs >> 2;
      sh = (uint32_t)(zs & 3) * 8u;
      z0 = zr[wi];
      z1 = zr[wi + 1 < rw ? wi + 1 : wi + 1 - rw];
      z2 = zr[wi + 2 < rw ? wi + 2 : wi + 2 - rw];
      z3 = zr[wi + 3 < rw ? wi + 3 : wi + 3 - rw];
      z4 = zr[wi + 4 < rw ? wi + 4 : wi + 4 - rw];
    }
    y0 = __funnelshift_r(z0, z1, sh);
    y1 = __funnelshift_r(z1, z2, sh);
    y2 = __funnelshift_r(z2, z3, sh);
    y3 = __funnelshift_r(z3, z4, sh);
  }
}

struct RoundArgs {
  Layout L;
  Tables tb;
  const uint8_t* in;
  long long in_stride;
  uint8_t* out;
  long long out_stride;
  const uint8_t* ks;
  long long ks_stride;
  const int* kmod;
  const uint8_t* agg_in;
  uint8_t* agg_out;
};

// Dynamic shared memory of an encryption round CTA:
// [tile Z, 16-aligned][the tile's keystream, T W C bytes when rows are whole
// 16-byte pieces, else none][sub-tile carries, NS bytes (per-channel chains:
// NS words) rounded to 16][share totals, 32 scan elements][row shifts, 32
// ints][the tile's subframe-start bit words][subframe seeds, SC bytes
// (per-channel: SC words)].  A decryption round uses the tile alone.
struct RoundSmem {
  int ks, carry, tot, kmod, sbits, seed, total;
  bool ks_staged;
};
__host__ __device__ inline RoundSmem round_smem(const Layout& L, bool pc = false) {
  RoundSmem m;
  const int rowb = L.W * L.C;
  const int w = pc ? 4 : 1;  // bytes per carry and per seed
  m.ks = (int)(((long long)L.T * tile_row_bytes(L.W, L.C) + 15) & ~15LL);
  m.ks_staged = (rowb & 15) == 0;
  m.carry = m.ks + (m.ks_staged ? L.T * rowb : 0);
  m.tot = m.carry + ((w * L.NS + 15) & ~15);
  m.kmod = m.tot + 32 * (pc ? 8 : 4);
  m.sbits = m.kmod + 32 * (int)sizeof(int);
  m.seed = m.sbits + 4 * (((L.T * L.W) >> 5) + 4);
  m.total = m.seed + w * L.SC;
  return m;
}

size_t round_smem_bytes(const Layout& L, bool pc) { return (size_t)round_smem(L, pc && L.C > 1).total; }
size_t dec_smem_bytes(const Layout& L) { return (size_t)(((long long)L.T * tile_row_bytes(L.W, L.C) + 15) & ~15LL); }

// 16-byte global -> shared copy that completes asynchronously (cp.async, L2
// only); cp_async_wait_all() waits for this thread's copies.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Byte qb of the current round's confused frame Y, read through Eq. 1 from
// the previous round's output X (with the pending sub-tile prefixes applied).
template <int C>
__device__ __forceinline__ uint8_t enc_y_at(const Layout& L, const Tables& tb, const uint8_t* X, const int* kmod,
                                            const uint8_t* s_carry, bool fix, int qb) {
  const int pp = qb / C, ch = qb - pp * C;
  const int alpha = pp / L.W, beta = pp - alpha * L.W;
  int o = beta - __ldg(&kmod[alpha]);
  if (o < 0) o += L.W;
  const int a = mod_h(alpha - o, L.H);
  const int qx = (a * L.W + o) * C + ch;
  uint8_t x = X[qx];
  if (fix) {
    const int sa = a >> L.lgR;
    if (qx < __ldg(&tb.fixlim[sa])) x ^= s_carry[sa];
  }
  return x;
}

// Pixel pp of the current round's confused frame Y as a word of C bytes (the
// per-channel seeds), read through Eq. 1 from the previous round's output X
// with the pending sub-tile word carries applied.
template <int C>
__device__ __forceinline__ uint32_t enc_ypx_at(const Layout& L, const Tables& tb, const uint8_t* X, const int* kmod,
                                               const uint32_t* s_carry, bool fix, int pp) {
  const int alpha = pp / L.W, beta = pp - alpha * L.W;
  int o = beta - __ldg(&kmod[alpha]);
  if (o < 0) o += L.W;
  const int a = mod_h(alpha - o, L.H);
  const int qx = (a * L.W + o) * C;
  uint32_t x = 0;
#pragma unroll
  for (int c = 0; c < C; c++) x |= (uint32_t)X[qx + c] << (8 * c);
  if (fix) {
    const int sa = a >> L.lgR;
    if (qx < __ldg(&tb.fixlim[sa])) x ^= s_carry[sa];
  }
  return x;
}

// Gather of the tile Z for C = 3 and 4 (T >= 4): each lane moves a run of
// four consecutive pixels of one source row (T / 4 lanes per source row), as
// four aligned 32-bit loads shifted into place and four 32-bit slot stores.
// Runs that wrap at H, leave the frame's columns or its bytes go pixel by
// pixel.  Z[tt][o] = X[(a0 + tt - o) mod H][o] as in the per-pixel gather.
// PC: the pending carries are pixel words (per-channel chains), else bytes.
template <int C, bool PC = false>
__device__ __forceinline__ void gather_runs(const Layout& L, const Tables& tb, const uint8_t* X, uint8_t* Z,
                                            const uint8_t* s_carry, const bool fix, const int a0, const int Te,
                                            const bool aligned) {
  constexpr int PR = 4;  // pixels per lane
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int LS = L.T / PR;  // lanes per source row
  const int rpw = 32 / LS;  // source rows per warp pass
  const int tt0 = (lane % LS) * PR;
  const int sub = lane / LS;
  const int astep = nw * rpw;
  const int MC = (L.W + L.H - 1) / L.H;
  uint32_t* Zw = reinterpret_cast<uint32_t*>(Z);
  constexpr int U = 4;  // source rows in flight per lane
  if (tt0 >= Te) return;
  const bool whole = tt0 + PR <= Te;
  for (int m = 0; m < MC; m++) {
    const int mo = m * L.H;
    for (int a = warp * rpw + sub; a < L.H; a += U * astep) {
      uint32_t w0[U], w1[U], w2[U], w3[U];
      int ov[U], qv[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int au = a + u * astep;
        int o = a0 + tt0 - au;
        if (o < 0) o += L.H;
        // the run's columns o .. o + 3 are consecutive, inside the frame and
        // its aligned words inside the frame's bytes
        const int qx = (au * L.W + o + mo) * C;
        const bool fast = aligned && whole && au < L.H && o + PR <= L.H && o + mo + PR <= L.W &&
                          (qx & ~3) + 16 <= L.N;
        ov[u] = au < L.H ? o + mo : -1;
        qv[u] = fast ? qx : -1;
        w0[u] = w1[u] = w2[u] = w3[u] = 0u;
        if (fast) {
          const uint32_t* src = reinterpret_cast<const uint32_t*>(X + (qx & ~3));
          w0[u] = __ldg(src);
          w1[u] = __ldg(src + 1);
          w2[u] = __ldg(src + 2);
          if (C == 4 || (qx & 3) != 0) w3[u] = __ldg(src + 3);
        }
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (ov[u] < 0) continue;
        const int au = a + u * astep;
        const int sa = au >> L.lgR;
        const int lim = fix ? __ldg(&tb.fixlim[sa]) : 0;
        const uint32_t cy =
            fix ? (PC ? reinterpret_cast<const uint32_t*>(s_carry)[sa] : rep_px<C>(s_carry[sa])) : 0u;
        if (qv[u] >= 0) {
          const int qx = qv[u];
          const uint32_t sh = (uint32_t)(qx & 3) * 8u;
          const uint32_t u0 = __funnelshift_r(w0[u], w1[u], sh), u1 = __funnelshift_r(w1[u], w2[u], sh);
          const uint32_t u2 = __funnelshift_r(w2[u], w3[u], sh), u3 = __funnelshift_r(w3[u], 0u, sh);
          uint32_t px[PR];
          if (C == 4) {
            px[0] = u0;
            px[1] = u1;
            px[2] = u2;
            px[3] = u3;
          } else {  // bytes 0-2, 3-5, 6-8, 9-11 of the run
            px[0] = u0 & 0xFFFFFFu;
            px[1] = __byte_perm(u0, u1, 0x0543u) & 0xFFFFFFu;
            px[2] = __byte_perm(u1, u2, 0x0432u) & 0xFFFFFFu;
            px[3] = u2 >> 8;
          }
#pragma unroll
          for (int j = 0; j < PR; j++) {
            uint32_t x = px[j];
            if (fix && qx + j * C < lim) x ^= cy;  // subframe starts are pixel-aligned
            Zw[zslot<C>(L, tt0 + j, ov[u] + j)] = x;
          }
        } else {
          // pixel by pixel: each tile row tt of the run has its own column
#pragma unroll
          for (int j = 0; j < PR; j++) {
            const int tt = tt0 + j;
            if (tt >= Te) break;
            int o = a0 + tt - au;
            if (o < 0) o += L.H;
            o += mo;
            if (o >= L.W) continue;
            const int qx = (au * L.W + o) * C;
            uint32_t x = load_px_g<C>(X, qx, aligned, L.N);
            if (fix && qx < lim) x ^= cy;
            Zw[zslot<C>(L, tt, o)] = x;
          }
        }
      }
    }
  }
}

// Diffusion of one warp's sub-tile (rows r0 .. r1 - 1) in chunks of 16
// pixels (16 C bytes) per lane, for C = 3 and 4 with W a multiple of 16 and
// the tile's keystream in shared memory (s_ks, tile byte offsets).  A chunk
// never crosses a row and, since the row rotation of Eq. 1 moves whole
// pixels, its source bytes in Z start at a pixel: sixteen slot loads packed
// into 4 C words.  The subframe starts of a chunk are 16 consecutive bits of
// one start-bit word.  Chunks with more than one start (or, without seed
// slots, any start) go byte by byte.
// c ? a : b, opaque to the compiler, so that a loop of selections over an
// unrolled register array stays in registers (an index would move the array
// to local memory).
__device__ __forceinline__ uint32_t sel_u32(bool c, uint32_t a, uint32_t b) {
  uint32_t r;
  asm("{\n .reg .pred p;\n setp.ne.u32 p, %3, 0;\n selp.b32 %0, %1, %2, p;\n}" : "=r"(r) : "r"(a), "r"(b),
      "r"((uint32_t)c));
  return r;
}

// Seed of the subframe starting at pixel pix (the rare many-starts path of
// diffuse_px16).
template <int C>
__device__ __forceinline__ uint8_t px16_seed(const RoundArgs& A, int pix, const uint32_t* s_sbits, int wlo,
                                          const uint8_t* s_seed, int s_lo, bool seeded, const uint8_t* X,
                                          const int* kmod, const uint8_t* s_carry, bool fix) {
  const Layout& L = A.L;
  const int wq = pix >> 5;
  const int s = __ldg(&A.tb.srank[wq]) + __popc(s_sbits[wq - wlo] & ((1u << (pix & 31)) - 1u));
  if (seeded) return s_seed[s - s_lo];
  const int nx = (s + 1 == L.n) ? 0 : s + 1;
  return enc_y_at<C>(L, A.tb, X, kmod, s_carry, fix, C * __ldg(&A.tb.pi[nx + 1]) - 1);
}

template <int C>
__device__ __forceinline__ void diffuse_px16(const RoundArgs& A, const int f, const uint8_t* Z, const uint8_t* s_ks,
                                             const int* s_kmod, const uint32_t* s_sbits, const int wlo,
                                             const uint8_t* s_seed, const int s_lo, const bool seeded,
                                             const uint8_t* X, const int* kmod, const uint8_t* s_carry,
                                             const bool fix, uint8_t* Out, const int a0, const int r0,
                                             const int r1) {
  constexpr int NW = 4 * C;  // words per chunk
  constexpr int CB = 16 * C;  // bytes per chunk
  const Layout& L = A.L;
  const int lane = threadIdx.x & 31;
  const int rowb = L.W * C;
  const int cpr = L.W >> 4;  // chunks per row
  const int nchunks = (r1 - r0) * cpr;
  const int tstart = a0 * rowb;
  const bool out_vec = ((reinterpret_cast<uintptr_t>(Out)) & 15) == 0;
  const uint32_t* Zw = reinterpret_cast<const uint32_t*>(Z);
  uint32_t run = 0;
  for (int cb = 0; cb < nchunks; cb += 32) {
    const int c = cb + lane;
    uint32_t pre[NW];
#pragma unroll
    for (int i = 0; i < NW; i++) pre[i] = 0u;
    int fse = CB;
    uint32_t agg = 0;
    int q0 = 0;
    if (c < nchunks) {
      const int rl = (c >= cpr ? 1 : 0) + (c >= 2 * cpr ? 1 : 0) + (c >= 3 * cpr ? 1 : 0);  // R <= 4
      const int p0 = (c - rl * cpr) << 4;  // first output pixel of the chunk in its row
      const int tt0 = r0 - a0 + rl;
      q0 = (r0 + rl) * rowb + p0 * C;  // first byte of the chunk in the frame
      int ps = p0 - s_kmod[tt0];       // first source pixel in the tile row (0 <= k < W)
      if (ps < 0) ps += L.W;
      const uint32_t* ksw = reinterpret_cast<const uint32_t*>(s_ks + (q0 - tstart));
      const int zb = tt0 * L.ZS;
      const bool contig = ps + 15 < L.W;  // the sixteen source pixels do not wrap at the row end
      const int s0 = zb + ps + (ps >> 5), lo = ps & 31;
      // slot of source pixel i (0..15) of the chunk
      auto slot = [&](int i) -> int {
        if (contig) return s0 + i + ((lo + i) >> 5);
        int q = ps + i;
        if (q >= L.W) q -= L.W;
        return zb + q + (q >> 5);
      };
      // packed word i (0..NW-1) of the chunk's source bytes, from its pixel slots
      auto yword = [&](int i) -> uint32_t {
        if (C == 4) return Zw[slot(i)];
        const int g = i / 3, r = i - 3 * g;  // word r of four 3-byte pixels 4g .. 4g + 3
        const uint32_t wa = Zw[slot(4 * g + r)], wb = Zw[slot(4 * g + r + 1)];
        return __byte_perm(wa, wb, r == 0 ? 0x4210u : (r == 1 ? 0x5421u : 0x6542u));
      };
      const int pix0 = (r0 + rl) * L.W + p0;  // a multiple of 16
      const uint32_t sw = (s_sbits[(pix0 >> 5) - wlo] >> (pix0 & 16)) & 0xFFFFu;
      const int nst = __popc(sw);
      if (nst == 0 || (nst == 1 && seeded)) {
        // d = b xor (y + b) per byte, its prefix XOR inside each word, then across words
#pragma unroll
        for (int i = 0; i < NW; i++) {
          const uint32_t kk = ksw[i];
          uint32_t d = kk ^ vadd4(yword(i), kk);
          d ^= d << 8;
          d ^= d << 16;
          if (i > 0) d ^= bcast3(pre[i - 1]);
          pre[i] = d;
        }
        if (nst == 1) {
          // byte kb starts subframe s: from kb on the chain is seed ^ d_kb ^ ..,
          // i.e. the chunk prefix xor (seed ^ prefix at kb - 1)
          const int b = __ffs(sw) - 1;
          const int kb = C * b;
          const int wq = pix0 >> 5;
          const int s = __ldg(&A.tb.srank[wq]) + __popc(s_sbits[wq - wlo] & ((1u << ((pix0 & 16) + b)) - 1u));
          uint32_t pk = 0;
          if (kb > 0) {
            const int km = kb - 1;
            uint32_t t = 0;
#pragma unroll
            for (int i = 0; i < NW; i++) t = sel_u32(i == (km >> 2), pre[i], t);
            pk = (t >> (8 * (km & 3))) & 0xFFu;
          }
          const uint32_t V = ((uint32_t)s_seed[s - s_lo] ^ pk) * 0x01010101u;
#pragma unroll
          for (int i = 0; i < NW; i++) pre[i] ^= V & mask_from(kb, 4 * i);
          fse = kb;
          agg = 0x100u | (pre[NW - 1] >> 24);
        } else {
          agg = pre[NW - 1] >> 24;
        }
      } else {
        // several starts in the chunk: byte by byte
        uint32_t v = 0;
        bool has = false;
#pragma unroll
        for (int i = 0; i < NW; i++) {
          const uint32_t yw = yword(i), kw = ksw[i];
          uint32_t o = 0;
#pragma unroll
          for (int bi = 0; bi < 4; bi++) {
            const int kb = 4 * i + bi;
            const uint8_t yb = (uint8_t)(yw >> (8 * bi));
            const uint8_t bb = (uint8_t)(kw >> (8 * bi));
            const uint8_t d = bb ^ (uint8_t)(yb + bb);
            if (kb % C == 0 && ((sw >> (kb / C)) & 1u)) {
              v = (uint32_t)(px16_seed<C>(A, pix0 + kb / C, s_sbits, wlo, s_seed, s_lo, seeded, X, kmod, s_carry,
                                          fix) ^ d);
              if (!has) {
                has = true;
                fse = kb;
              }
            } else {
              v ^= d;
            }
            o |= (v & 0xFFu) << (8 * bi);
          }
          pre[i] = o;
        }
        agg = (has ? 0x100u : 0u) | (v & 0xFFu);
      }
    }
    // warp-wide segmented scan of the chunks' values, then the running carry
    const uint32_t incl = warp_incl_scan(agg);
    uint32_t excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
    if (lane == 0) excl = 0;
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint32_t E = seg_combine(run, excl);
    run = seg_combine(run, total);
    if (c < nchunks) {
      const uint32_t evx4 = (E & 0xFFu) * 0x01010101u;
      if (fse == CB) {
#pragma unroll
        for (int i = 0; i < NW; i++) pre[i] ^= evx4;
      } else {
#pragma unroll
        for (int i = 0; i < NW; i++) pre[i] ^= evx4 & ~mask_from(fse, 4 * i);  // bytes before fse miss E
      }
      if (out_vec) {
        uint4* o4 = reinterpret_cast<uint4*>(Out + q0);
#pragma unroll
        for (int i = 0; i < NW / 4; i++) o4[i] = make_uint4(pre[4 * i], pre[4 * i + 1], pre[4 * i + 2], pre[4 * i + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < NW; i++) {
#pragma unroll
          for (int bi = 0; bi < 4; bi++) Out[q0 + 4 * i + bi] = (uint8_t)(pre[i] >> (8 * bi));
        }
      }
    }
  }
  if (lane == 0) A.agg_out[(long long)f * L.NS + (r0 >> L.lgR)] = (uint8_t)run;
}

// ---- per-channel chains (the alternative reading of Eq. 3: byte ch of pixel
// p follows byte ch of pixel p - 1 of the subframe) --------------------------
// The scan runs over pixel words: d_p = b_p xor (y_p + b_p) byte by byte, the
// chain value c_p = c_{p-1} xor d_p, reset to seed xor d_p at a subframe start
// (seed = the confused pixel at the end of the next subframe).  Sub-tile
// carries and aggregates are pixel words; otherwise the tile, the lazy
// carries and the fix-up are those of the byte chains.

// Keystream bytes of pixel j (0..15) of a 16-pixel chunk held as 4 C packed
// words kw (j a compile-time index).
template <int C>
__device__ __forceinline__ uint32_t chunk_px(const uint32_t* kw, int j) {
  if (C == 4) return kw[j];
  const int g = j >> 2, r = j & 3;
  const uint32_t u0 = kw[3 * g], u1 = kw[3 * g + 1], u2 = kw[3 * g + 2];
  return r == 0 ? (u0 & 0xFFFFFFu)
                : (r == 1 ? (__byte_perm(u0, u1, 0x0543u) & 0xFFFFFFu)
                          : (r == 2 ? (__byte_perm(u1, u2, 0x0432u) & 0xFFFFFFu) : (u2 >> 8)));
}

// Seed pixel of the subframe starting at pixel pix.
template <int C>
__device__ __forceinline__ uint32_t pc_seed_at(const RoundArgs& A, int pix, const uint32_t* s_sbits, int wlo,
                                               const uint32_t* s_seed, int s_lo, bool seeded, const uint8_t* X,
                                               const int* kmod, const uint32_t* s_carry, bool fix) {
  const int wq = pix >> 5;
  const int s = __ldg(&A.tb.srank[wq]) + __popc(s_sbits[wq - wlo] & ((1u << (pix & 31)) - 1u));
  if (seeded) return s_seed[s - s_lo];
  const int nx = (s + 1 == A.L.n) ? 0 : s + 1;
  return enc_ypx_at<C>(A.L, A.tb, X, kmod, s_carry, fix, __ldg(&A.tb.pi[nx + 1]) - 1);
}

// The warp's sub-tile (rows r0 .. r1 - 1) in chunks of 16 pixels per lane,
// for W a multiple of 16 with the tile's keystream in shared memory: sixteen
// pixel slots and 4 C keystream words in, 4 C packed words out (16-byte
// stores).  Chunks with more than one subframe start (or, without seed slots,
// any) take their seeds one by one.
template <int C>
__device__ __forceinline__ void diffuse_pc16(const RoundArgs& A, const int f, const uint8_t* Z, const uint8_t* s_ks,
                                             const int* s_kmod, const uint32_t* s_sbits, const int wlo,
                                             const uint32_t* s_seed, const int s_lo, const bool seeded,
                                             const uint8_t* X, const int* kmod, const uint32_t* s_carry,
                                             const bool fix, uint8_t* Out, const int a0, const int r0,
                                             const int r1) {
  constexpr int NW = 4 * C;  // words per chunk
  using T = CarryT<true>;
  const Layout& L = A.L;
  const int lane = threadIdx.x & 31;
  const int rowb = L.W * C;
  const int cpr = L.W >> 4;  // chunks per row
  const int nchunks = (r1 - r0) * cpr;
  const int tstart = a0 * rowb;
  const bool out_vec = ((reinterpret_cast<uintptr_t>(Out)) & 15) == 0;
  const uint32_t* Zw = reinterpret_cast<const uint32_t*>(Z);
  uint64_t run = 0;
  for (int cb = 0; cb < nchunks; cb += 32) {
    const int c = cb + lane;
    uint32_t px[16];
#pragma unroll
    for (int j = 0; j < 16; j++) px[j] = 0u;
    int fse = 16;
    uint64_t agg = 0;
    int q0 = 0;
    if (c < nchunks) {
      const int rl = (c >= cpr ? 1 : 0) + (c >= 2 * cpr ? 1 : 0) + (c >= 3 * cpr ? 1 : 0);  // R <= 4
      const int p0 = (c - rl * cpr) << 4;  // first output pixel of the chunk in its row
      const int tt0 = r0 - a0 + rl;
      q0 = (r0 + rl) * rowb + p0 * C;  // first byte of the chunk in the frame
      int ps = p0 - s_kmod[tt0];       // first source pixel in the tile row
      if (ps < 0) ps += L.W;
      const uint32_t* ksw = reinterpret_cast<const uint32_t*>(s_ks + (q0 - tstart));
      const int zb = tt0 * L.ZS;
      const bool contig = ps + 15 < L.W;
      const int s0 = zb + ps + (ps >> 5), lo = ps & 31;
      auto slot = [&](int i) -> int {
        if (contig) return s0 + i + ((lo + i) >> 5);
        int q = ps + i;
        if (q >= L.W) q -= L.W;
        return zb + q + (q >> 5);
      };
      uint32_t kw[NW];
#pragma unroll
      for (int i = 0; i < NW; i++) kw[i] = ksw[i];
      const int pix0 = (r0 + rl) * L.W + p0;  // a multiple of 16
      const uint32_t sw = (s_sbits[(pix0 >> 5) - wlo] >> (pix0 & 16)) & 0xFFFFu;
      const int nst = __popc(sw);
      if (nst == 0 || (nst == 1 && seeded)) {
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < 16; j++) {
          const uint32_t b = chunk_px<C>(kw, j);
          acc ^= b ^ vadd4(Zw[slot(j)], b);
          px[j] = acc;
        }
        if (nst == 1) {
          // pixel j0 starts subframe s: from j0 on the chain is seed ^ d_j0 ^ ..,
          // i.e. the chunk prefix xor (seed ^ prefix at j0 - 1)
          const int j0 = __ffs(sw) - 1;
          const int wq = pix0 >> 5;
          const int s = __ldg(&A.tb.srank[wq]) + __popc(s_sbits[wq - wlo] & ((1u << ((pix0 & 16) + j0)) - 1u));
          uint32_t pk = 0;
#pragma unroll
          for (int j = 0; j < 15; j++) pk = sel_u32(j == j0 - 1, px[j], pk);
          const uint32_t V = s_seed[s - s_lo] ^ pk;
#pragma unroll
          for (int j = 0; j < 16; j++) px[j] ^= sel_u32(j >= j0, V, 0u);
          fse = j0;
          agg = T::F | px[15];
        } else {
          agg = px[15];
        }
      } else {
        uint32_t v = 0;
        bool has = false;
#pragma unroll
        for (int j = 0; j < 16; j++) {
          const uint32_t b = chunk_px<C>(kw, j);
          const uint32_t d = b ^ vadd4(Zw[slot(j)], b);
          if ((sw >> j) & 1u) {
            v = pc_seed_at<C>(A, pix0 + j, s_sbits, wlo, s_seed, s_lo, seeded, X, kmod, s_carry, fix) ^ d;
            if (!has) {
              has = true;
              fse = j;
            }
          } else {
            v ^= d;
          }
          px[j] = v;
        }
        agg = (has ? T::F : 0ull) | v;
      }
    }
    // warp-wide segmented scan of the chunks' values, then the running carry
    const uint64_t incl = warp_scan_t<true>(agg);
    uint64_t excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
    if (lane == 0) excl = 0;
    const uint64_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint64_t E = seg_comb<true>(run, excl);
    run = seg_comb<true>(run, total);
    if (c < nchunks) {
      const uint32_t ev = (uint32_t)E;
#pragma unroll
      for (int j = 0; j < 16; j++) px[j] ^= sel_u32(j < fse, ev, 0u);  // pixels before fse miss E
      uint32_t ow[NW];
      if (C == 4) {
#pragma unroll
        for (int j = 0; j < 16; j++) ow[j] = px[j];
      } else {
#pragma unroll
        for (int g = 0; g < 4; g++) {
          ow[3 * g] = px[4 * g] | (px[4 * g + 1] << 24);
          ow[3 * g + 1] = (px[4 * g + 1] >> 8) | (px[4 * g + 2] << 16);
          ow[3 * g + 2] = (px[4 * g + 2] >> 16) | (px[4 * g + 3] << 8);
        }
      }
      if (out_vec) {
        uint4* o4 = reinterpret_cast<uint4*>(Out + q0);
#pragma unroll
        for (int i = 0; i < NW / 4; i++) o4[i] = make_uint4(ow[4 * i], ow[4 * i + 1], ow[4 * i + 2], ow[4 * i + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < NW; i++) {
#pragma unroll
          for (int bi = 0; bi < 4; bi++) Out[q0 + 4 * i + bi] = (uint8_t)(ow[i] >> (8 * bi));
        }
      }
    }
  }
  if (lane == 0) reinterpret_cast<uint32_t*>(A.agg_out)[(long long)f * L.NS + (r0 >> L.lgR)] = (uint32_t)run;
}

// Any other shape: 16 consecutive pixels of the sub-tile per lane, one pixel
// at a time (slot, keystream bytes, start bit), bytes stored one by one.
template <int C>
__device__ __forceinline__ void diffuse_pc_any(const RoundArgs& A, const int f, const uint8_t* Z, const uint8_t* s_ks,
                                               const bool ks_staged, const uint8_t* KS, const int* s_kmod,
                                               const uint32_t* s_sbits, const int wlo, const uint32_t* s_seed,
                                               const int s_lo, const bool seeded, const uint8_t* X, const int* kmod,
                                               const uint32_t* s_carry, const bool fix, uint8_t* Out, const int a0,
                                               const int r0, const int r1) {
  using T = CarryT<true>;
  const Layout& L = A.L;
  const int lane = threadIdx.x & 31;
  const int pbeg = r0 * L.W, pend = r1 * L.W;
  const int tstart = a0 * L.W * C;
  const int nchunks = (pend - pbeg + 15) >> 4;
  const uint32_t* Zw = reinterpret_cast<const uint32_t*>(Z);
  uint64_t run = 0;
  for (int cb = 0; cb < nchunks; cb += 32) {
    const int c = cb + lane;
    const int q = pbeg + 16 * c;
    const int len = c < nchunks ? min(16, pend - q) : 0;
    uint32_t px[16];
#pragma unroll
    for (int j = 0; j < 16; j++) px[j] = 0u;
    int fse = 16;
    uint64_t agg = 0;
    if (len > 0) {
      int row = q / L.W;
      int beta = q - row * L.W;
      uint32_t v = 0;
      bool has = false;
#pragma unroll
      for (int j = 0; j < 16; j++) {
        if (j < len) {
          const int p = q + j;
          const int tt = row - a0;
          int zo = beta - s_kmod[tt];
          if (zo < 0) zo += L.W;
          const uint32_t y = Zw[zslot<C>(L, tt, zo)];
          uint32_t b = 0;
#pragma unroll
          for (int ch = 0; ch < C; ch++)
            b |= (uint32_t)(ks_staged ? s_ks[p * C - tstart + ch] : KS[p * C + ch]) << (8 * ch);
          const uint32_t d = b ^ vadd4(y, b);
          if ((s_sbits[(p >> 5) - wlo] >> (p & 31)) & 1u) {
            v = pc_seed_at<C>(A, p, s_sbits, wlo, s_seed, s_lo, seeded, X, kmod, s_carry, fix) ^ d;
            if (!has) {
              has = true;
              fse = j;
            }
          } else {
            v ^= d;
          }
          px[j] = v;
          if (++beta == L.W) {
            beta = 0;
            row++;
          }
        }
      }
      agg = (has ? T::F : 0ull) | v;
    }
    const uint64_t incl = warp_scan_t<true>(agg);
    uint64_t excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
    if (lane == 0) excl = 0;
    const uint64_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint64_t E = seg_comb<true>(run, excl);
    run = seg_comb<true>(run, total);
    if (len > 0) {
      const uint32_t ev = (uint32_t)E;
#pragma unroll
      for (int j = 0; j < 16; j++) {
        if (j < len) {
          const uint32_t o = px[j] ^ (j < fse ? ev : 0u);
#pragma unroll
          for (int ch = 0; ch < C; ch++) Out[(q + j) * C + ch] = (uint8_t)(o >> (8 * ch));
        }
      }
    }
  }
  if (lane == 0) reinterpret_cast<uint32_t*>(A.agg_out)[(long long)f * L.NS + (r0 >> L.lgR)] = (uint32_t)run;
}

// PC: per-channel chains (C = 3 or 4), else chains over the subframe's bytes.
template <int C, bool PC = false>
__device__ __forceinline__ void enc_round_tile(const RoundArgs& A, const int f, const int t, uint8_t* smem) {
  static_assert(!PC || C > 1, "per-channel chains with one channel are the byte chains");
  const Layout& L = A.L;
  const int rowb = L.W * C;
  const int a0 = t * L.T;
  const int Te = min(L.T, L.H - a0);
  const RoundSmem sm = round_smem(L, PC);
  uint8_t* Z = smem;
  uint8_t* s_carry = smem + sm.carry;
  uint32_t* s_tot = reinterpret_cast<uint32_t*>(smem + sm.tot);
  int* s_kmod = reinterpret_cast<int*>(smem + sm.kmod);
  uint32_t* s_sbits = reinterpret_cast<uint32_t*>(smem + sm.sbits);
  uint8_t* s_seed = smem + sm.seed;
  const uint8_t* s_ks = smem + sm.ks;

  const uint8_t* X = A.in + f * A.in_stride;
  uint8_t* Out = A.out + f * A.out_stride;
  const uint8_t* KS = A.ks + f * A.ks_stride;
  const int* kmod = A.kmod + (long long)f * L.H;
  const bool fix = A.agg_in != nullptr;
  // subframes s_lo .. s_hi - 1 start in this tile's pixels
  const int s_lo = starts_before(L, a0 * L.W), s_hi = starts_before(L, (a0 + Te) * L.W);
  const bool seeded = L.SC > 0;
  // start-bit words wlo .. wlo + nsw - 1 cover the tile's pixels and one word more
  const int wlo = (a0 * L.W) >> 5;
  const int nsw = ((((a0 + Te) * L.W - 1) >> 5) + 1) - wlo + 1;

  // the tile's keystream (bytes [tstart, tstart + Te W C) of the round) into
  // shared memory, in flight while the carries, seeds and gather run
  const int tstart = a0 * rowb;
  const bool ks_staged = sm.ks_staged && ((reinterpret_cast<uintptr_t>(KS + tstart) & 15) == 0);
  if (ks_staged) {
    const int n16 = (Te * rowb) >> 4;
    for (int k = threadIdx.x; k < n16; k += blockDim.x) cp_async16(smem + sm.ks + 16 * k, KS + tstart + 16 * k);
    cp_async_commit();
  }
  uint32_t* s_carry_w = reinterpret_cast<uint32_t*>(s_carry);
  uint32_t* s_seed_w = reinterpret_cast<uint32_t*>(s_seed);
  if (fix) {
    if constexpr (PC)
      sub_carries_t<true>(L, A.tb, reinterpret_cast<const uint32_t*>(A.agg_in) + (long long)f * L.NS, s_carry_w,
                          reinterpret_cast<uint64_t*>(s_tot));
    else
      sub_carries(L, A.tb, A.agg_in + (long long)f * L.NS, s_carry, s_tot);
  }
  if (threadIdx.x < Te) s_kmod[threadIdx.x] = kmod[a0 + threadIdx.x];
  for (int k = threadIdx.x; k < nsw; k += blockDim.x) s_sbits[k] = __ldg(&A.tb.sbits[wlo + k]);
  __syncthreads();

  // ---- seeds (Eq. 3 with the seed of reading R9) of the subframes starting
  // here: the pre-diffusion byte at the end of the next subframe, read
  // through Eq. 1 from the previous round's output
  if (seeded) {
    for (int k = threadIdx.x; k < s_hi - s_lo; k += blockDim.x) {
      const int s = s_lo + k;
      const int nx = (s + 1 == L.n) ? 0 : s + 1;
      if constexpr (PC)
        s_seed_w[k] = enc_ypx_at<C>(L, A.tb, X, kmod, s_carry_w, fix, __ldg(&A.tb.pi[nx + 1]) - 1);
      else
        s_seed[k] = enc_y_at<C>(L, A.tb, X, kmod, s_carry, fix, C * __ldg(&A.tb.pi[nx + 1]) - 1);
    }
  }

  // ---- gather: Z[tt][o] = X[(a0 + tt - o) mod H][o] -------------------------
  if constexpr (C == 3 || C == 4) {
    if (L.T >= 4)
      gather_runs<C, PC>(L, A.tb, X, Z, s_carry, fix, a0, Te, (reinterpret_cast<uintptr_t>(X) & 3) == 0);
  }
  if (C == 1 || L.T < 4) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rpw = 32 / L.T;  // source rows per warp pass
    const int tt = lane & (L.T - 1);
    const int sub = lane / L.T;
    const int astep = nw * rpw;
    const int MC = (L.W + L.H - 1) / L.H;  // columns o, o + H, ... of a source row per tile row
    const bool aligned = (reinterpret_cast<uintptr_t>(X) & 3) == 0;
    constexpr int U = 8;  // source rows in flight per lane
    if (tt < Te) {
      for (int m = 0; m < MC; m++) {
        const int mo = m * L.H;
        for (int a = warp * rpw + sub; a < L.H; a += U * astep) {
          uint32_t v[U];
          int zo[U];
#pragma unroll
          for (int u = 0; u < U; u++) {
            const int au = a + u * astep;
            int o = a0 + tt - au;
            if (o < 0) o += L.H;
            o += mo;
            zo[u] = (au < L.H && o < L.W) ? o : -1;
            v[u] = zo[u] >= 0 ? load_px_g<C>(X, (au * L.W + o) * C, aligned, L.N) : 0u;
          }
#pragma unroll
          for (int u = 0; u < U; u++) {
            if (zo[u] < 0) continue;
            uint32_t x = v[u];
            if (fix) {
              const int au = a + u * astep;
              const int sa = au >> L.lgR;
              // subframe starts are pixel-aligned: the whole pixel is on one side of fixlim
              if ((au * L.W + zo[u]) * C < __ldg(&A.tb.fixlim[sa]))
                x ^= PC ? s_carry_w[sa] : rep_px<C>(s_carry[sa]);
            }
            store_z<C>(Z, zslot<C>(L, tt, zo[u]), x);
          }
        }
      }
    }
  }
  if (ks_staged) cp_async_wait_all();
  __syncthreads();

  // ---- diffusion of this warp's sub-tile, 16-byte chunks per lane ------------
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int WPT = L.T >> L.lgR;  // sub-tiles per tile
  const int r0 = a0 + warp * L.R;
  if (warp >= WPT || r0 >= a0 + Te) return;
  const int r1 = min(r0 + L.R, a0 + Te);
  if constexpr (PC) {
    if (ks_staged && (L.W & 15) == 0)
      diffuse_pc16<C>(A, f, Z, s_ks, s_kmod, s_sbits, wlo, s_seed_w, s_lo, seeded, X, kmod, s_carry_w, fix, Out, a0,
                      r0, r1);
    else
      diffuse_pc_any<C>(A, f, Z, s_ks, ks_staged, KS, s_kmod, s_sbits, wlo, s_seed_w, s_lo, seeded, X, kmod,
                        s_carry_w, fix, Out, a0, r0, r1);
    return;
  }
  if constexpr (C == 3 || C == 4) {
    if (ks_staged && (L.W & 15) == 0) {
      diffuse_px16<C>(A, f, Z, s_ks, s_kmod, s_sbits, wlo, s_seed, s_lo, seeded, X, kmod, s_carry, fix, Out, a0, r0,
                      r1);
      return;
    }
  }
  const int ws = r0 * rowb, we = r1 * rowb;
  const int base16 = ws & ~15;
  const int nchunks = (we - base16 + 15) >> 4;
  const bool out_vec = ((reinterpret_cast<uintptr_t>(Out)) & 15) == 0;
  uint32_t run = 0;
  // keystream of the lane's next full chunk (shared memory when staged, else
  // global memory one iteration ahead)
  auto ks_full = [&](int cc) -> uint4 {
    const int s0 = base16 + 16 * cc;
    if (cc < nchunks && s0 >= ws && s0 + 16 <= we)
      return ks_staged ? *reinterpret_cast<const uint4*>(s_ks + (s0 - tstart))
                       : *reinterpret_cast<const uint4*>(KS + s0);
    return make_uint4(0u, 0u, 0u, 0u);
  };
  uint4 kv_next = ks_full(lane);
  for (int cb = 0; cb < nchunks; cb += 32) {
    const int c = cb + lane;
    const uint4 kv = kv_next;
    kv_next = ks_full(c + 32);
    int cs = base16 + 16 * c, ce = cs + 16;
    if (cs < ws) cs = ws;
    if (ce > we) ce = we;
    const int len = (c < nchunks && ce > cs) ? ce - cs : 0;
    uint32_t pre[4] = {0u, 0u, 0u, 0u};
    int fse = 16;
    uint32_t agg = 0;
    bool fast = false;
    if (len == 16 && (cs & 15) == 0) {
      // fast path: the chunk lies in one row (for C = 1: its rotated source
      // bytes do not wrap, or the row is whole words) and at most one subframe
      // starts inside it (its seed is in shared memory)
      const int rloc = cs - ws;  // < R rows (R <= 4)
      const int rl = (rloc >= rowb ? 1 : 0) + (rloc >= 2 * rowb ? 1 : 0) + (rloc >= 3 * rowb ? 1 : 0);
      const int tt0 = r0 - a0 + rl;
      const int e0 = rloc - rl * rowb;
      int zs = e0 - s_kmod[tt0] * C;
      if (zs < 0) zs += rowb;
      if (e0 + 16 <= rowb && (C != 1 || zs + 16 <= rowb || (rowb & 3) == 0)) {
        const int pfirst = (cs + C - 1) / C, plast = (cs + 15) / C;
        const int wq = pfirst >> 5;
        const uint64_t win = (uint64_t)s_sbits[wq - wlo] | ((uint64_t)s_sbits[wq - wlo + 1] << 32);
        const int lb = pfirst - (wq << 5), hb = plast - (wq << 5);
        const uint64_t sw = win & ((2ull << hb) - 1ull) & ~((1ull << lb) - 1ull);
        const int nst = __popcll(sw);
        if (nst == 0 || (nst == 1 && seeded)) {
          fast = true;
          uint32_t y0, y1, y2, y3;
          z_row16<C>(L, Z, tt0, zs, y0, y1, y2, y3);
          uint32_t d0 = kv.x ^ vadd4(y0, kv.x), d1 = kv.y ^ vadd4(y1, kv.y);
          uint32_t d2 = kv.z ^ vadd4(y2, kv.z), d3 = kv.w ^ vadd4(y3, kv.w);
          d0 ^= d0 << 8;
          d0 ^= d0 << 16;
          d1 ^= d1 << 8;
          d1 ^= d1 << 16;
          d2 ^= d2 << 8;
          d2 ^= d2 << 16;
          d3 ^= d3 << 8;
          d3 ^= d3 << 16;
          d1 ^= bcast3(d0);
          d2 ^= bcast3(d1);
          d3 ^= bcast3(d2);
          if (nst == 1) {
            // byte k starts subframe s: from k on the chain is seed ^ d_k ^ ..,
            // i.e. the chunk prefix xor (seed ^ prefix at k - 1); bytes before
            // k still miss the incoming prefix
            const int b = __ffsll((long long)sw) - 1;
            const int k = C * ((wq << 5) + b) - cs;
            const int s = __ldg(&A.tb.srank[wq]) + __popcll(win & ((1ull << b) - 1ull));
            uint32_t pk = 0;
            if (k > 0) {
              const int km = k - 1;
              const uint32_t wsel = km < 4 ? d0 : (km < 8 ? d1 : (km < 12 ? d2 : d3));
              pk = (wsel >> (8 * (km & 3))) & 0xFFu;
            }
            const uint32_t V = ((uint32_t)s_seed[s - s_lo] ^ pk) * 0x01010101u;
            d0 ^= V & mask_from(k, 0);
            d1 ^= V & mask_from(k, 4);
            d2 ^= V & mask_from(k, 8);
            d3 ^= V & mask_from(k, 12);
            fse = k;
            agg = 0x100u | (d3 >> 24);
          } else {
            agg = d3 >> 24;
          }
          pre[0] = d0;
          pre[1] = d1;
          pre[2] = d2;
          pre[3] = d3;
        }
      }
    }
    if (len > 0 && !fast) {
      uint8_t kb[16];
#pragma unroll
      for (int k = 0; k < 16; k++) kb[k] = k < len ? (ks_staged ? s_ks[cs - tstart + k] : KS[cs + k]) : 0;
      const int off = cs - tstart;
      int tt = off / rowb;
      int e = off - tt * rowb;
      int beta = e / C;
      int ch = e - beta * C;
      int zo = beta - s_kmod[tt];
      if (zo < 0) zo += L.W;
      const int pix0 = cs / C;
      const int w0 = pix0 >> 5;
      const uint64_t win = (uint64_t)s_sbits[w0 - wlo] | ((uint64_t)s_sbits[w0 - wlo + 1] << 32);
      uint32_t v = 0;
      bool has = false;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        if (k < len) {
          const uint8_t y = z_byte<C>(L, Z, tt, zo, ch);
          const uint8_t b = kb[k];
          const uint8_t d = b ^ (uint8_t)(y + b);
          bool st = false;
          int pix = 0;
          if (ch == 0) {
            pix = (cs + k) / C;
            st = (win >> (pix - (w0 << 5))) & 1ull;
          }
          if (st) {
            const int wq = pix >> 5;
            const int s = __ldg(&A.tb.srank[wq]) + __popc(s_sbits[wq - wlo] & ((1u << (pix & 31)) - 1u));
            uint8_t sd;
            if (seeded) {
              sd = s_seed[s - s_lo];
            } else {
              const int nx = (s + 1 == L.n) ? 0 : s + 1;
              sd = enc_y_at<C>(L, A.tb, X, kmod, s_carry, fix, C * __ldg(&A.tb.pi[nx + 1]) - 1);
            }
            v = (uint32_t)(sd ^ d);
            if (!has) {
              has = true;
              fse = k;
            }
          } else {
            v ^= d;
          }
          pre[k >> 2] |= (v & 0xFFu) << (8 * (k & 3));
          if (++ch == C) {
            ch = 0;
            if (++zo == L.W) zo = 0;
          }
          if (++e == rowb) {
            e = 0;
            ch = 0;
            tt++;
            if (tt < Te) {
              zo = L.W - s_kmod[tt];
              if (zo == L.W) zo = 0;
            }
          }
        }
      }
      agg = (has ? 0x100u : 0u) | (v & 0xFFu);
    }
    // warp-wide segmented scan of the chunks' values, then the running carry
    const uint32_t incl = warp_incl_scan(agg);
    uint32_t excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
    if (lane == 0) excl = 0;
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint32_t E = seg_combine(run, excl);
    run = seg_combine(run, total);
    if (len > 0) {
      const uint32_t evx4 = (E & 0xFFu) * 0x01010101u;
#pragma unroll
      for (int w4 = 0; w4 < 4; w4++) pre[w4] ^= evx4 & ~mask_from(fse, 4 * w4);  // bytes before fse miss E
      if (len == 16 && (cs & 15) == 0 && out_vec) {
        *reinterpret_cast<uint4*>(Out + cs) = make_uint4(pre[0], pre[1], pre[2], pre[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 16; k++)
          if (k < len) Out[cs + k] = (uint8_t)(pre[k >> 2] >> (8 * (k & 3)));
      }
    }
  }
  if (lane == 0) A.agg_out[(long long)f * L.NS + (r0 >> L.lgR)] = (uint8_t)run;
}

template <int C, bool PC>
__global__ void __launch_bounds__(kRoundThreads, 3) k_enc_round(RoundArgs A) {
  extern __shared__ __align__(16) uint8_t smem[];
  enc_round_tile<C, PC>(A, blockIdx.y, blockIdx.x, smem);
}

template <int C, bool PC>
static cudaError_t enc_round_c(const RoundArgs& A, int nframes, cudaStream_t st) {
  const size_t smem = round_smem_bytes(A.L, PC);
  cudaError_t e = allow_smem(k_enc_round<C, PC>, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(A.L.NT, nframes);
  k_enc_round<C, PC><<<grid, kRoundThreads, smem, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_enc_round(const Layout& L, Tables tb, const uint8_t* in, long long in_stride, uint8_t* out,
                             long long out_stride, const uint8_t* ks_round, long long ks_stride, const int* kmod,
                             const uint8_t* agg_in, uint8_t* agg_out, int nframes, cudaStream_t st, bool pc) {
  if (nframes <= 0) return cudaSuccess;
  RoundArgs A{L, tb, in, in_stride, out, out_stride, ks_round, ks_stride, kmod, agg_in, agg_out};
  switch (L.C) {
    case 1: return enc_round_c<1, false>(A, nframes, st);
    case 3: return pc ? enc_round_c<3, true>(A, nframes, st) : enc_round_c<3, false>(A, nframes, st);
    case 4: return pc ? enc_round_c<4, true>(A, nframes, st) : enc_round_c<4, false>(A, nframes, st);
  }
  return cudaErrorInvalidValue;
}

// Shared memory of the fix-up: the carries (NS bytes, or NS words for
// per-channel chains, rounded to 16) and the carry scan's share totals (32
// scan elements).
__host__ __device__ inline int fixup_smem_bytes(const Layout& L, bool pc = false) {
  return pc ? ((4 * L.NS + 15) & ~15) + 32 * 8 : ((L.NS + 15) & ~15) + 32 * 4;
}

// After the last round: apply each sub-tile's missing prefix in place (one warp
// per sub-tile of tile t).
__device__ __forceinline__ void enc_fixup_tile(const Layout& L, const Tables& tb, uint8_t* out, long long out_stride,
                                               const uint8_t* agg, const int f, const int t, uint8_t* smem) {
  uint8_t* s_carry = smem;
  sub_carries(L, tb, agg + (long long)f * L.NS, s_carry, reinterpret_cast<uint32_t*>(smem + ((L.NS + 15) & ~15)));
  const int rowb = L.W * L.C;
  uint8_t* O = out + f * out_stride;
  const int lane = threadIdx.x & 31;
  const int WPT = L.T >> L.lgR;
  for (int w = threadIdx.x >> 5; w < WPT; w += blockDim.x >> 5) {
    const int s = t * WPT + w;
    if (s == 0 || s >= L.NS) continue;
    const int sstart = s * L.R * rowb;
    const int lim = __ldg(&tb.fixlim[s]);
    if (lim <= sstart) continue;
    const uint8_t cy = s_carry[s];
    const uint32_t c4 = cy * 0x01010101u;
    // head bytes up to 16-byte alignment, aligned body, tail bytes
    const uintptr_t addr = reinterpret_cast<uintptr_t>(O + sstart);
    int head = (int)((16 - (addr & 15)) & 15);
    if (head > lim - sstart) head = lim - sstart;
    if (lane < head) O[sstart + lane] ^= cy;
    const int body0 = sstart + head;
    const int nvec = (lim - body0) >> 4;
    uint4* V = reinterpret_cast<uint4*>(O + body0);
    for (int k = lane; k < nvec; k += 32) {
      uint4 v = V[k];
      v.x ^= c4;
      v.y ^= c4;
      v.z ^= c4;
      v.w ^= c4;
      V[k] = v;
    }
    for (int k = body0 + nvec * 16 + lane; k < lim; k += 32) O[k] ^= cy;
  }
}

// The same for per-channel chains: the missing prefix is a pixel word, XORed
// into the C bytes of every pixel before the sub-tile's first subframe start.
__device__ __forceinline__ void enc_fixup_tile_pc(const Layout& L, const Tables& tb, uint8_t* out,
                                                  long long out_stride, const uint8_t* agg, const int f, const int t,
                                                  uint8_t* smem) {
  uint32_t* s_carry = reinterpret_cast<uint32_t*>(smem);
  sub_carries_t<true>(L, tb, reinterpret_cast<const uint32_t*>(agg) + (long long)f * L.NS, s_carry,
                      reinterpret_cast<uint64_t*>(smem + ((4 * L.NS + 15) & ~15)));
  const int C = L.C;
  uint8_t* O = out + f * out_stride;
  const int lane = threadIdx.x & 31;
  const int WPT = L.T >> L.lgR;
  for (int w = threadIdx.x >> 5; w < WPT; w += blockDim.x >> 5) {
    const int s = t * WPT + w;
    if (s == 0 || s >= L.NS) continue;
    const int p0 = s * L.R * L.W;               // first pixel of the sub-tile
    const int p1 = __ldg(&tb.fixlim[s]) / C;    // its first subframe start (pixel-aligned) or its end
    const uint32_t cy = s_carry[s];
    if (cy == 0u) continue;
    for (int p = p0 + lane; p < p1; p += 32) {
#pragma unroll 4
      for (int ch = 0; ch < C; ch++) O[p * C + ch] ^= (uint8_t)(cy >> (8 * ch));
    }
  }
}

__global__ void __launch_bounds__(kRoundThreads) k_enc_fixup(Layout L, Tables tb, uint8_t* out, long long out_stride,
                                                             const uint8_t* agg) {
  extern __shared__ __align__(16) uint8_t smem[];
  enc_fixup_tile(L, tb, out, out_stride, agg, blockIdx.y, blockIdx.x, smem);
}

__global__ void __launch_bounds__(kRoundThreads) k_enc_fixup_pc(Layout L, Tables tb, uint8_t* out,
                                                                long long out_stride, const uint8_t* agg) {
  extern __shared__ __align__(16) uint8_t smem[];
  enc_fixup_tile_pc(L, tb, out, out_stride, agg, blockIdx.y, blockIdx.x, smem);
}

cudaError_t launch_enc_fixup(const Layout& L, Tables tb, uint8_t* out, long long out_stride, const uint8_t* agg,
                             int nframes, cudaStream_t st, bool pc) {
  if (nframes <= 0) return cudaSuccess;
  pc = pc && L.C > 1;
  const int smem = fixup_smem_bytes(L, pc);
  cudaError_t e = pc ? allow_smem(k_enc_fixup_pc, smem) : allow_smem(k_enc_fixup, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(L.NT, nframes);
  if (pc)
    k_enc_fixup_pc<<<grid, kRoundThreads, smem, st>>>(L, tb, out, out_stride, agg);
  else
    k_enc_fixup<<<grid, kRoundThreads, smem, st>>>(L, tb, out, out_stride, agg);
  return cudaGetLastError();
}

// Byte-wise a - b mod 256 in each of the eight bytes of a word.
__device__ __forceinline__ uint64_t vsub8(uint64_t a, uint64_t b) {
  constexpr uint64_t Hb = 0x8080808080808080ull;
  return ((a | Hb) - (b & ~Hb)) ^ ((a ^ ~b) & Hb);
}

// Decryption round (Eq. 4 then Eq. 2), one CTA per (row band of the output
// frame X, frame): X[a][o] = Y[alpha][beta] with alpha = (a + o) mod H and
// beta = (o + k(alpha)) mod W, where y_q = ((b ^ c_q ^ c_{q-1}) - b) mod 256 and,
// at a subframe start, c_{q-1} is replaced by the seed: the decrypted byte at
// the end of the next subframe (reading R10; never itself a start, S_i >= 2).
// Band row tt takes one pixel from every ciphertext row (o = alpha - a0 - tt
// mod H, + m H), so the lanes of a warp read runs of consecutive pixels of a
// row.  Eight rows are handled per iteration in phases (row shifts, then
// ciphertext, keystream and start-bit words, then the result) so that a lane
// keeps several rows of loads in flight; each decrypted pixel is one 32-bit
// shared-memory slot (C = 3, 4), packed into bytes when the band is written.
// PC: per-channel chains (C = 3 or 4): c_{q-1} is then the same byte of the
// previous pixel, and the seed the decrypted last pixel of the next subframe.
template <int C, int U = 4, bool PC = false>
__device__ __forceinline__ void dec_round_tile(const RoundArgs& A, const int f, const int t, uint8_t* smem) {
  static_assert(!PC || C > 1, "per-channel chains with one channel are the byte chains");
  const Layout& L = A.L;
  const int rowb = L.W * C;
  const int a0 = t * L.T;
  const int Te = min(L.T, L.H - a0);
  uint8_t* Xt = smem;
  const uint8_t* Cin = A.in + f * A.in_stride;
  uint8_t* Out = A.out + f * A.out_stride;
  const uint8_t* KS = A.ks + f * A.ks_stride;
  const int* kmod = A.kmod + (long long)f * L.H;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rpw = 32 / L.T;
  const int tt = lane & (L.T - 1);
  const int sub = lane / L.T;
  const int astep = nw * rpw;
  const uint32_t pmask = C == 4 ? 0xFFFFFFFFu : ((1u << (8 * C)) - 1u);
  // the decrypted pixel at pixel index pix of the round's input, byte by byte
  auto cpx = [&](const uint8_t* base, int pp) -> uint32_t {  // the C bytes of pixel pp
    uint32_t v = 0;
#pragma unroll
    for (int c = 0; c < C; c++) v |= (uint32_t)base[pp * C + c] << (8 * c);
    return v;
  };
  auto decrypt_pixel = [&](int pix, uint32_t sw) -> uint32_t {
    const int qb = pix * C;
    if constexpr (PC) {
      uint32_t prev;
      if ((sw >> (pix & 31)) & 1u) {  // subframe start: the seed pixel
        const int s = __ldg(&A.tb.srank[pix >> 5]) + __popc(sw & ((1u << (pix & 31)) - 1u));
        const int nx = (s + 1 == L.n) ? 0 : s + 1;
        const int sp = __ldg(&A.tb.pi[nx + 1]) - 1;
        const uint32_t bs = cpx(KS, sp);
        prev = vsub4(bs ^ cpx(Cin, sp) ^ cpx(Cin, sp - 1), bs) & pmask;
      } else {
        prev = cpx(Cin, pix - 1);
      }
      const uint32_t b = cpx(KS, pix);
      return vsub4(b ^ cpx(Cin, pix) ^ prev, b) & pmask;
    }
    uint8_t prev;
    if ((sw >> (pix & 31)) & 1u) {  // subframe start: the seed
      const int s = __ldg(&A.tb.srank[pix >> 5]) + __popc(sw & ((1u << (pix & 31)) - 1u));
      const int nx = (s + 1 == L.n) ? 0 : s + 1;
      const int sb = C * __ldg(&A.tb.pi[nx + 1]) - 1;
      const uint8_t bs = KS[sb];
      prev = (uint8_t)((uint8_t)(bs ^ Cin[sb] ^ Cin[sb - 1]) - bs);
    } else {
      prev = Cin[qb - 1];
    }
    uint32_t v = 0;
#pragma unroll
    for (int c = 0; c < C; c++) {
      const uint8_t cq = Cin[qb + c];
      const uint8_t b = KS[qb + c];
      v |= (uint32_t)(uint8_t)((uint8_t)(b ^ cq ^ prev) - b) << (8 * c);
      prev = cq;
    }
    return v;
  };
  // ciphertext bytes q-1 .. q+C-1 and keystream bytes q .. q+C-1 of a pixel as
  // two aligned words each (frame bases 4-byte aligned, away from the frame
  // ends); bytes one by one otherwise
  const bool words = ((reinterpret_cast<uintptr_t>(Cin) | reinterpret_cast<uintptr_t>(KS)) & 3) == 0;
  const int MC = (L.W + L.H - 1) / L.H;
  if (tt < Te) {
    for (int m = 0; m < MC; m++) {
      const int mo = m * L.H;
      for (int alpha = warp * rpw + sub; alpha < L.H; alpha += U * astep) {
        int pix[U], ov[U];
        uint32_t c0[U], c1[U], c2[U], k0[U], k1[U], sw[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int al = alpha + u * astep;
          int o = al - (a0 + tt);
          if (o < 0) o += L.H;
          o += mo;
          ov[u] = (al < L.H && o < L.W) ? o : -1;
          int beta = 0;
          if (ov[u] >= 0) {
            beta = o + __ldg(&kmod[al]);
            if (beta >= L.W) beta -= L.W;
          }
          pix[u] = al * L.W + beta;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int qb = pix[u] * C;
          sw[u] = ov[u] >= 0 ? __ldg(&A.tb.sbits[pix[u] >> 5]) : 0u;  // start bits, with the data
          c2[u] = 0;
          if (PC && ov[u] >= 0 && words && qb >= C && qb + 12 <= L.N) {
            // ciphertext bytes qb - C .. qb + C - 1 (three words), keystream qb .. qb + C - 1
            const uint32_t* cw = reinterpret_cast<const uint32_t*>(Cin + ((qb - C) & ~3));
            const uint32_t* kw = reinterpret_cast<const uint32_t*>(KS + (qb & ~3));
            c0[u] = __ldg(cw);
            c1[u] = __ldg(cw + 1);
            c2[u] = C == 3 ? __ldg(cw + 2) : 0u;
            k0[u] = __ldg(kw);
            k1[u] = C == 3 ? __ldg(kw + 1) : 0u;
          } else if (!PC && ov[u] >= 0 && words && qb >= 4 && qb + 8 <= L.N) {
            const uint32_t* cw = reinterpret_cast<const uint32_t*>(Cin + ((qb - 1) & ~3));
            const uint32_t* kw = reinterpret_cast<const uint32_t*>(KS + (qb & ~3));
            c0[u] = __ldg(cw);
            c1[u] = __ldg(cw + 1);
            k0[u] = __ldg(kw);
            k1[u] = __ldg(kw + 1);
          } else {
            c0[u] = c1[u] = k0[u] = k1[u] = 0;
          }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
          if (ov[u] < 0) continue;
          const int p = pix[u], qb = p * C;
          uint32_t y;
          const bool fast = PC ? (words && qb >= C && qb + 12 <= L.N) : (words && qb >= 4 && qb + 8 <= L.N);
          if (((sw[u] >> (p & 31)) & 1u) || !fast) {
            y = decrypt_pixel(p, sw[u]);
          } else if constexpr (PC) {
            uint32_t prev, cur, b;
            if (C == 4) {  // qb is a multiple of 4
              prev = c0[u];
              cur = c1[u];
              b = k0[u];
            } else {
              const uint32_t sh = (uint32_t)((qb - 3) & 3) * 8u;
              const uint32_t lo = __funnelshift_r(c0[u], c1[u], sh), hi = __funnelshift_r(c1[u], c2[u], sh);
              prev = lo & 0xFFFFFFu;
              cur = __byte_perm(lo, hi, 0x0543u) & 0xFFFFFFu;
              b = __funnelshift_r(k0[u], k1[u], (uint32_t)(qb & 3) * 8u) & 0xFFFFFFu;
            }
            y = vsub4(b ^ cur ^ prev, b) & pmask;
          } else {
            const uint64_t c = ((uint64_t)c1[u] << 32 | c0[u]) >> (8 * ((qb - 1) & 3));
            const uint64_t b = ((uint64_t)k1[u] << 32 | k0[u]) >> (8 * (qb & 3));
            y = (uint32_t)vsub8(b ^ (c >> 8) ^ c, b) & pmask;
          }
          store_z<C>(Xt, zslot<C>(L, tt, ov[u]), y);
        }
      }
    }
  }
  __syncthreads();
  // write the band's rows (contiguous bytes of the output frame)
  const int tstart = a0 * rowb;
  const int nb = Te * rowb;
  uint8_t* dstg = Out + tstart;
  if (C == 1) {
    if ((reinterpret_cast<uintptr_t>(dstg) & 15) == 0) {
      const int nvec = nb >> 4;
      for (int k = threadIdx.x; k < nvec; k += blockDim.x)
        reinterpret_cast<uint4*>(dstg)[k] = reinterpret_cast<const uint4*>(Xt)[k];
      for (int k = nvec * 16 + threadIdx.x; k < nb; k += blockDim.x) dstg[k] = Xt[k];
    } else {
      for (int k = threadIdx.x; k < nb; k += blockDim.x) dstg[k] = Xt[k];
    }
    return;
  }
  // 16-byte chunks at 16-byte frame offsets: whole chunks inside one row are
  // packed from six (C = 3) or four (C = 4) pixel slots, the others byte by byte
  const bool out_vec = (reinterpret_cast<uintptr_t>(Out) & 15) == 0;
  const int base16 = tstart & ~15;
  const int tend = tstart + nb;
  const int nchunks = (tend - base16 + 15) >> 4;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x) {
    int cs = base16 + 16 * c, ce = cs + 16;
    if (cs < tstart) cs = tstart;
    if (ce > tend) ce = tend;
    const int off = cs - tstart;
    const int r = off / rowb;
    const int e0 = off - r * rowb;
    if (ce - cs == 16 && (cs & 15) == 0 && e0 + 16 <= rowb) {
      uint32_t y0, y1, y2, y3;
      z_row16<C>(L, Xt, r, e0, y0, y1, y2, y3);
      if (out_vec) {
        *reinterpret_cast<uint4*>(Out + cs) = make_uint4(y0, y1, y2, y3);
      } else {
        const uint32_t yw[4] = {y0, y1, y2, y3};
#pragma unroll
        for (int k = 0; k < 16; k++) Out[cs + k] = (uint8_t)(yw[k >> 2] >> (8 * (k & 3)));
      }
    } else {
      for (int q = cs; q < ce; q++) {
        const int oq = q - tstart;
        const int rr = oq / rowb, e = oq - rr * rowb;
        const int px = e / C;
        Out[q] = z_byte<C>(L, Xt, rr, px, e - px * C);
      }
    }
  }
}

// Decryption round in scatter form (C = 3 or 4, W a multiple of 16, rows of
// whole 16-byte pieces, 16-byte aligned frames): one CTA per band of rows of
// the round's INPUT, the ciphertext C.  Eq. 4 is elementwise (each byte needs
// c_q, c_{q-1} or, per channel, c_{q-C}, and b_q), so the band is read
// contiguously, 16 pixels per lane and step (C 16-byte loads of ciphertext and
// of keystream plus the word before), decrypted with byte-wise SWAR into the
// band's pixel slots in shared memory, and then written through Eq. 2:
// Y[alpha][beta] goes to X[a][o] with o = (beta - k(alpha)) mod W and
// a = (alpha - o) mod H, so output row a receives the T consecutive columns
// o = alpha - a (mod H, + m H) from the band's T rows.  Four lanes write one
// output row's run (4 pixels each), realigned by a shuffle so that every
// 32-bit store is aligned and inside the run; the run's first and last partial
// words go byte by byte (their other bytes belong to neighbouring bands).
// Subframe starts use the decrypted seed at the end of the next subframe.
template <int C, bool PC>
__device__ __forceinline__ void dec_scatter_tile(const RoundArgs& A, const int f, const int t, uint8_t* smem) {
  constexpr int NW = 4 * C;       // words per 16-pixel unit
  constexpr int CS = PC ? C : 1;  // the chain's step in bytes
  const Layout& L = A.L;
  const int a0 = t * L.T;
  const int Te = min(L.T, L.H - a0);
  uint32_t* Yw = reinterpret_cast<uint32_t*>(smem);
  int* s_kmod = reinterpret_cast<int*>(smem + (((long long)L.T * tile_row_bytes(L.W, C) + 15) & ~15LL));
  const uint8_t* Cin = A.in + f * A.in_stride;
  uint8_t* Out = A.out + f * A.out_stride;
  const uint8_t* KS = A.ks + f * A.ks_stride;
  const int* kmod = A.kmod + (long long)f * L.H;
  if (threadIdx.x == 0) {
    // the band's ciphertext and keystream towards L2 ahead of the unit loads
    // (band starts and sizes are multiples of 16 bytes)
    const long long qb = (long long)a0 * L.W * C;
    const uint32_t nb = (uint32_t)(Te * L.W * C);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(Cin + qb), "r"(nb) : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(KS + qb), "r"(nb) : "memory");
  }
  if (threadIdx.x < Te) s_kmod[threadIdx.x] = __ldg(&kmod[a0 + threadIdx.x]);
  auto cpx = [&](const uint8_t* base, int pp) -> uint32_t {  // the C bytes of pixel pp
    uint32_t v = 0;
#pragma unroll
    for (int c = 0; c < C; c++) v |= (uint32_t)__ldg(base + pp * C + c) << (8 * c);
    return v;
  };
  const uint32_t pmask = C == 4 ? 0xFFFFFFFFu : 0xFFFFFFu;

  // ---- Eq. 4 over the band, 16 pixels per lane and step ---------------------
  const int upr = L.W >> 4;  // units per row
  const int nunits = Te * upr;
  for (int u = threadIdx.x; u < nunits; u += blockDim.x) {
    const int rl = u / upr;
    const int beta0 = (u - rl * upr) << 4;
    const int p0 = (a0 + rl) * L.W + beta0;
    const int q0 = p0 * C;  // a multiple of 16
    uint32_t c[NW + 1], b[NW];  // c[0]: the ciphertext word before the unit
    c[0] = q0 > 0 ? __ldg(reinterpret_cast<const uint32_t*>(Cin + q0) - 1) : 0u;
#pragma unroll
    for (int i = 0; i < C; i++) {
      const uint4 x = __ldg(reinterpret_cast<const uint4*>(Cin + q0) + i);
      const uint4 y = __ldg(reinterpret_cast<const uint4*>(KS + q0) + i);
      c[1 + 4 * i] = x.x;
      c[2 + 4 * i] = x.y;
      c[3 + 4 * i] = x.z;
      c[4 + 4 * i] = x.w;
      b[4 * i] = y.x;
      b[4 * i + 1] = y.y;
      b[4 * i + 2] = y.z;
      b[4 * i + 3] = y.w;
    }
    uint32_t yv[NW];
#pragma unroll
    for (int i = 0; i < NW; i++) {
      // ciphertext bytes q - CS of the word's bytes q
      const uint32_t prev = CS == 4 ? c[i] : __funnelshift_r(c[i], c[i + 1], 32 - 8 * CS);
      yv[i] = vsub4(b[i] ^ c[i + 1] ^ prev, b[i]);
    }
    const uint32_t sw = (__ldg(&A.tb.sbits[p0 >> 5]) >> (p0 & 16)) & 0xFFFFu;
    if (sw != 0u) {
      // pixels that start a subframe: their first byte (per channel: all C
      // bytes) follows the decrypted seed at the end of the next subframe
#pragma unroll
      for (int j = 0; j < 16; j++) {
        if ((sw >> j) & 1u) {
          const int pix = p0 + j;
          const int s = __ldg(&A.tb.srank[pix >> 5]) +
                        __popc(__ldg(&A.tb.sbits[pix >> 5]) & ((1u << (pix & 31)) - 1u));
          const int nx = (s + 1 == L.n) ? 0 : s + 1;
          const int sp = __ldg(&A.tb.pi[nx + 1]) - 1;  // never a start: every subframe has 2 bytes or more
          if constexpr (PC) {
            const uint32_t bs = cpx(KS, sp);
            const uint32_t seed = vsub4(bs ^ cpx(Cin, sp) ^ cpx(Cin, sp - 1), bs) & pmask;
            const uint32_t bb = cpx(KS, pix), cc = cpx(Cin, pix);
            const uint32_t v = vsub4(bb ^ cc ^ seed, bb) & pmask;
#pragma unroll
            for (int ch = 0; ch < C; ch++) {
              const int k = j * C + ch;  // byte of the unit (compile-time)
              const uint32_t sh = 8u * (uint32_t)(k & 3);
              yv[k >> 2] = (yv[k >> 2] & ~(0xFFu << sh)) | (((v >> (8 * ch)) & 0xFFu) << sh);
            }
          } else {
            const int sb = sp * C + C - 1;  // the last byte of subframe nx
            const uint8_t bs = __ldg(KS + sb);
            const uint8_t seed = (uint8_t)((uint8_t)(bs ^ __ldg(Cin + sb) ^ __ldg(Cin + sb - 1)) - bs);
            const int k = j * C;
            const uint32_t sh = 8u * (uint32_t)(k & 3);
            const uint8_t bb = (uint8_t)(b[k >> 2] >> sh), cc = (uint8_t)(c[1 + (k >> 2)] >> sh);
            const uint8_t v = (uint8_t)((uint8_t)(bb ^ cc ^ seed) - bb);
            yv[k >> 2] = (yv[k >> 2] & ~(0xFFu << sh)) | ((uint32_t)v << sh);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 16; j++) Yw[zslot<C>(L, rl, beta0 + j)] = C == 4 ? yv[j] : chunk_px<C>(yv, j);
  }
  __syncthreads();

  // ---- Eq. 2: runs of the band's columns into the output rows ---------------
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int MC = (L.W + L.H - 1) / L.H;
  const bool full = Te == L.T && L.T >= 4;
  if (full) {
    const int LS = L.T / 4;  // lanes per output row (4 pixels each)
    const int rpw = 32 / LS;
    const int tt0 = (lane % LS) * 4;
    const int k = lane % LS;  // the lane's segment in its row's run
    const int sub = lane / LS;
    for (int m = 0; m < MC; m++) {
      const int mo = m * L.H;
      for (int abase = warp * rpw; abase < L.H; abase += nw * rpw) {  // warp-uniform trips
        const int a = abase + sub;
        int os = a0 - a;  // column of band row 0 in output row a (mod H)
        if (os < 0) os += L.H;
        // the row's run is contiguous, inside the frame's columns: aligned stores
        const bool fast = a < L.H && os + L.T <= L.H && os + mo + L.T <= L.W;
        uint32_t px[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int tt = tt0 + j;
          int o = os + tt;
          if (o >= L.H) o -= L.H;
          o += mo;
          int beta = o + s_kmod[tt];
          if (beta >= L.W) beta -= L.W;
          px[j] = (a < L.H && o < L.W) ? Yw[tt * L.ZS + beta + (beta >> 5)] : 0u;
        }
        if (C == 4) {
          if (fast) {
            uint32_t* dst = reinterpret_cast<uint32_t*>(Out + ((long long)a * L.W + os + mo + tt0) * 4);
#pragma unroll
            for (int j = 0; j < 4; j++) dst[j] = px[j];
            continue;
          }
        } else {
          // the lane's 12 bytes as three words, and the next lane's first word
          const uint32_t w0 = px[0] | (px[1] << 24), w1 = (px[1] >> 8) | (px[2] << 16);
          const uint32_t w2 = (px[2] >> 16) | (px[3] << 8);
          const uint32_t n0 = __shfl_down_sync(0xFFFFFFFFu, w0, 1);
          if (fast) {
            const long long S = ((long long)a * L.W + os + mo + tt0) * 3;  // the segment's first byte
            const int r = (int)(S & 3);
            const int sh = (4 - r) & 3;  // bytes up to the first aligned word
            uint32_t* dst = reinterpret_cast<uint32_t*>(Out + S + sh);
            const uint32_t v0 = __funnelshift_r(w0, w1, 8 * sh), v1 = __funnelshift_r(w1, w2, 8 * sh);
            const uint32_t v2 = __funnelshift_r(w2, n0, 8 * sh);
            if (k == 0) {  // the run's head bytes
              for (int i = 0; i < sh; i++) Out[S + i] = (uint8_t)(w0 >> (8 * i));
            }
            dst[0] = v0;
            dst[1] = v1;
            if (k < LS - 1 || r == 0) {
              dst[2] = v2;
            } else {  // the run's tail: r bytes of the last word are ours
              for (int i = 0; i < r; i++) Out[S + sh + 8 + i] = (uint8_t)(v2 >> (8 * i));
            }
            continue;
          }
        }
        // pixel by pixel (the run wraps at H or leaves the frame's columns)
        if (a < L.H) {
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const int tt = tt0 + j;
            int o = os + tt;
            if (o >= L.H) o -= L.H;
            o += mo;
            if (o >= L.W) continue;
            uint8_t* d = Out + ((long long)a * L.W + o) * C;
#pragma unroll
            for (int c2 = 0; c2 < C; c2++) d[c2] = (uint8_t)(px[j] >> (8 * c2));
          }
        }
      }
    }
  } else {
    // a partial band or fewer than 4 rows: pixel by pixel, one band row per lane
    for (int m = 0; m < MC; m++) {
      const int mo = m * L.H;
      for (int idx = threadIdx.x; idx < L.H * Te; idx += blockDim.x) {
        const int a = idx / Te, tt = idx - a * Te;
        int o = a0 + tt - a;
        if (o < 0) o += L.H;
        o += mo;
        if (o >= L.W) continue;
        int beta = o + s_kmod[tt];
        if (beta >= L.W) beta -= L.W;
        const uint32_t v = Yw[tt * L.ZS + beta + (beta >> 5)];
        uint8_t* d = Out + ((long long)a * L.W + o) * C;
#pragma unroll
        for (int c2 = 0; c2 < C; c2++) d[c2] = (uint8_t)(v >> (8 * c2));
      }
    }
  }
}

template <int C, bool PC>
__global__ void __launch_bounds__(kRoundThreads, 4) k_dec_scatter(RoundArgs A) {
  extern __shared__ __align__(16) uint8_t smem[];
  dec_scatter_tile<C, PC>(A, blockIdx.y, blockIdx.x, smem);
}

template <int C, bool PC>
__global__ void __launch_bounds__(kRoundThreads, 4) k_dec_round(RoundArgs A) {
  extern __shared__ __align__(16) uint8_t smem[];
  dec_round_tile<C, 4, PC>(A, blockIdx.y, blockIdx.x, smem);
}

template <int C, bool PC>
static cudaError_t dec_round_c(const RoundArgs& A, int nframes, cudaStream_t st) {
  const Layout& L = A.L;
  dim3 grid(L.NT, nframes);
  // the scatter form when the band can be read as whole 16-byte pieces and the
  // output rows written as aligned words (and input and output are apart)
  const uintptr_t al = reinterpret_cast<uintptr_t>(A.in) | reinterpret_cast<uintptr_t>(A.ks) |
                       reinterpret_cast<uintptr_t>(A.out) | (uintptr_t)A.in_stride | (uintptr_t)A.ks_stride |
                       (uintptr_t)A.out_stride;
  const bool apart = A.in + (long long)(nframes - 1) * A.in_stride + L.N <= A.out ||
                     A.out + (long long)(nframes - 1) * A.out_stride + L.N <= A.in;
  if constexpr (C > 1) {
    if ((L.W & 15) == 0 && (al & 15) == 0 && apart) {
      const size_t smem = dec_smem_bytes(L) + 32 * sizeof(int);
      cudaError_t e = allow_smem(k_dec_scatter<C, PC>, (int)smem);
      if (e != cudaSuccess) return e;
      k_dec_scatter<C, PC><<<grid, kRoundThreads, smem, st>>>(A);
      return cudaGetLastError();
    }
  }
  const size_t smem = dec_smem_bytes(L);
  cudaError_t e = allow_smem(k_dec_round<C, PC>, (int)smem);
  if (e != cudaSuccess) return e;
  k_dec_round<C, PC><<<grid, kRoundThreads, smem, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_dec_round(const Layout& L, Tables tb, const uint8_t* in, long long in_stride, uint8_t* out,
                             long long out_stride, const uint8_t* ks_round, long long ks_stride, const int* kmod,
                             int nframes, cudaStream_t st, bool pc) {
  if (nframes <= 0) return cudaSuccess;
  RoundArgs A{L, tb, in, in_stride, out, out_stride, ks_round, ks_stride, kmod, nullptr, nullptr};
  switch (L.C) {
    case 1: return dec_round_c<1, false>(A, nframes, st);
    case 3: return pc ? dec_round_c<3, true>(A, nframes, st) : dec_round_c<3, false>(A, nframes, st);
    case 4: return pc ? dec_round_c<4, true>(A, nframes, st) : dec_round_c<4, false>(A, nframes, st);
  }
  return cudaErrorInvalidValue;
}

// =============================================================================
// Ragged batch: many streams, frames, resolutions and both directions in one
// launch per phase (schedule, shift tables, keystream, each round, fix-up).
// The round kernels are persistent: a grid sized to the GPU walks the
// batch-wide (job, frame, tile) list.
// =============================================================================

// largest j < nj with key(J[j]) <= x (keys are non-decreasing)
template <typename Key>
__device__ __forceinline__ int find_job(const JobDesc* J, int nj, int x, Key key) {
  int lo = 0, hi = nj - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key(J[mid]) <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Jobs of mode 1 only consume keystream produced earlier into their ring;
// the host gives them no keystream or shift-table work (zero-length ranges).
__global__ void k_batch_sc(const JobDesc* J, const BatchHdr* hdr) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < hdr->njobs && J[j].nframes > 0 && J[j].mode != 1)
    frame_sc_serial(J[j].main, J[j].nframes, J[j].sc, J[j].ring_cap, J[j].ring_slot0);
}

__device__ __forceinline__ int job_slot(const JobDesc& d, int f) {
  return d.ring_cap > 0 ? (d.ring_slot0 + f) % d.ring_cap : f;
}

__global__ void k_batch_kmod(const JobDesc* J, const BatchHdr* hdr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= hdr->total_kmod) return;
  const int j = find_job(J, hdr->njobs, idx, [](const JobDesc& d) { return d.kmod_base; });
  const JobDesc& d = J[j];
  const int local = idx - d.kmod_base;
  const int f = local / d.L.H;
  const int a = local - f * d.L.H;
  const int slot = job_slot(d, f);
  d.kmod[(long long)slot * d.L.H + a] = kmod_of(d.L, d.sc[slot], a);
}

__global__ void __launch_bounds__(32) k_batch_ks(const JobDesc* J, const BatchHdr* hdr) {
  const int w = blockIdx.x;
  if (w >= hdr->total_warps) return;
  const int j = find_job(J, hdr->njobs, w, [](const JobDesc& d) { return d.warp_base; });
  const JobDesc& d = J[j];
  const int i = (w - d.warp_base) * 16 + (threadIdx.x >> 1);
  const int side = threadIdx.x & 1;
  if (d.kind == 0)
    ks_plcm_fx_chain(d.L, d.tb, d.ch, d.nframes, d.ks, i, side, d.ring_cap, d.ring_slot0);
  else if (d.kind == 2)
    ks_pair_chain<2, false>(d.L, d.tb, d.ch, d.nframes, d.ks, i, side, d.ring_cap, d.ring_slot0);
  else if (d.sine_b64)
    ks_pair_chain<1, false, true>(d.L, d.tb, d.ch, d.nframes, d.ks, i, side, d.ring_cap, d.ring_slot0);
  else
    ks_pair_chain<1, false>(d.L, d.tb, d.ch, d.nframes, d.ks, i, side, d.ring_cap, d.ring_slot0);
}

// The same over CTAs of W warps that each hold a whole SM (their dynamic shared
// memory is claimed, not used): for the batch's long chains, which bound the
// batch and lose issue slots when other chains or round CTAs share their SM.
template <int W>
__global__ void __launch_bounds__(W * 32) k_batch_ks_sm(const JobDesc* J, const BatchHdr* hdr) {
  const int w = blockIdx.x * W + (threadIdx.x >> 5);
  if (w >= hdr->total_warps) return;
  const int lane = threadIdx.x & 31;
  const int j = find_job(J, hdr->njobs, w, [](const JobDesc& d) { return d.warp_base; });
  const JobDesc& d = J[j];
  const int i = (w - d.warp_base) * 16 + (lane >> 1);
  const int side = lane & 1;
  if (d.kind == 0)
    ks_plcm_fx_chain(d.L, d.tb, d.ch, d.nframes, d.ks, i, side, d.ring_cap, d.ring_slot0);
  else if (d.kind == 2)
    ks_pair_chain<2, false>(d.L, d.tb, d.ch, d.nframes, d.ks, i, side, d.ring_cap, d.ring_slot0);
  else if (d.sine_b64)
    ks_pair_chain<1, false, true>(d.L, d.tb, d.ch, d.nframes, d.ks, i, side, d.ring_cap, d.ring_slot0);
  else
    ks_pair_chain<1, false>(d.L, d.tb, d.ch, d.nframes, d.ks, i, side, d.ring_cap, d.ring_slot0);
}

// Round `step` of frame f of a job (job rounds may differ): encryption applies
// round `step`, decryption round r - 1 - step; the buffers alternate as in a
// single-stream pass.  Every pointer is offset to frame f.
__device__ __forceinline__ RoundArgs batch_round_args(const JobDesc& d, int step, int f) {
  const Layout& L = d.L;
  const int r = L.rounds;
  const int jr = d.dir == 0 ? step : r - 1 - step;
  const int slot = job_slot(d, f);
  RoundArgs A{};
  A.L = L;
  A.tb = d.tb;
  A.in_stride = step == 0 ? (long long)L.N : L.Npad;
  A.in = (step == 0 ? d.in : d.buf[(step - 1) & 1]) + f * A.in_stride;
  A.out_stride = step == r - 1 ? (long long)L.N : L.Npad;
  A.out = (step == r - 1 ? d.out : d.buf[step & 1]) + f * A.out_stride;
  A.ks = d.ks + (long long)slot * r * L.Npad + (long long)jr * L.Npad;
  A.ks_stride = 0;
  A.kmod = d.kmod + (long long)slot * L.H;
  const long long aw = d.pc ? 4 : 1;  // bytes per sub-tile aggregate
  A.agg_in = (d.dir == 0 && step > 0) ? d.agg[(step - 1) & 1] + (long long)f * L.NS * aw : nullptr;
  A.agg_out = d.dir == 0 ? d.agg[step & 1] + (long long)f * L.NS * aw : nullptr;
  return A;
}

// One round of every tile of the batch's jobs of one (direction, channels,
// chains) variant: their tiles are the contiguous range [vbeg, vend) (jobs
// ordered by variant), so each variant is a lean kernel like the single-stream
// ones.
template <int DIR, int C, bool PC = false>
__global__ void __launch_bounds__(kRoundThreads, 3) k_batch_round(const JobDesc* J, const BatchHdr* hdr, int step) {
  extern __shared__ __align__(16) uint8_t smem[];
  // the item's round arguments, built once per CTA and read by every thread as
  // shared-memory broadcasts (a per-thread copy would live in local memory)
  __shared__ RoundArgs sA;
  __shared__ int s_item[3];  // the round applies, tile, decryption in scatter form
  constexpr int v = DIR * 5 + (C == 1 ? 0 : (C == 3 ? 1 : 2)) + (PC ? 2 : 0);
  const int beg = hdr->vbeg[v], end = hdr->vend[v], nj = hdr->njobs;
  for (int item = beg + blockIdx.x; item < end; item += gridDim.x) {
    if (threadIdx.x == 0) {
      const int j = find_job(J, nj, item, [](const JobDesc& d) { return d.tile_base; });
      const JobDesc& d = J[j];
      s_item[0] = step < d.L.rounds;
      if (step < d.L.rounds) {
        const int local = item - d.tile_base;
        const int f = local / d.L.NT;
        s_item[1] = local - f * d.L.NT;
        sA = batch_round_args(d, step, f);
        // the scatter form (as for a single stream): rows of whole 16-byte
        // pieces, 16-byte aligned frames, input and output apart
        const uintptr_t al = reinterpret_cast<uintptr_t>(sA.in) | reinterpret_cast<uintptr_t>(sA.ks) |
                             reinterpret_cast<uintptr_t>(sA.out);
        s_item[2] = DIR == 1 && C > 1 && (d.L.W & 15) == 0 && (al & 15) == 0 &&
                    (sA.in + d.L.N <= sA.out || sA.out + d.L.N <= sA.in);
      }
    }
    __syncthreads();
    if (s_item[0]) {
      if (DIR == 0) {
        enc_round_tile<C, PC>(sA, 0, s_item[1], smem);
      } else {
        if constexpr (C > 1) {
          if (s_item[2])
            dec_scatter_tile<C, PC>(sA, 0, s_item[1], smem);
          else
            dec_round_tile<C, 4, PC>(sA, 0, s_item[1], smem);
        } else {
          dec_round_tile<C, 4, PC>(sA, 0, s_item[1], smem);
        }
      }
    }
    __syncthreads();  // shared memory (and sA) is reused by the next item
  }
}

template <int DIR, int C, bool PC = false>
static cudaError_t batch_round_attr(size_t smem) {
  return allow_smem(k_batch_round<DIR, C, PC>, (int)smem);
}

template <int DIR, int C, bool PC = false>
static cudaError_t batch_round_ctas(size_t smem, int* ctas) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_batch_round<DIR, C, PC>, kRoundThreads, smem);
}

__global__ void __launch_bounds__(kRoundThreads) k_batch_fixup(const JobDesc* J, const BatchHdr* hdr) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int total = hdr->total_tiles, nj = hdr->njobs;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = find_job(J, nj, item, [](const JobDesc& d) { return d.tile_base; });
    const JobDesc& d = J[j];
    if (d.dir == 0) {
      const int local = item - d.tile_base;
      const int f = local / d.L.NT;
      const int t = local - f * d.L.NT;
      if (d.pc)
        enc_fixup_tile_pc(d.L, d.tb, d.out, d.L.N, d.agg[(d.L.rounds - 1) & 1], f, t, smem);
      else
        enc_fixup_tile(d.L, d.tb, d.out, d.L.N, d.agg[(d.L.rounds - 1) & 1], f, t, smem);
    }
    __syncthreads();
  }
}

cudaError_t prepare_batch_kernels(size_t smem) {
  cudaError_t e = allow_smem(k_batch_fixup, (int)smem);
  if (e == cudaSuccess) e = batch_round_attr<0, 1>(smem);
  if (e == cudaSuccess) e = batch_round_attr<0, 3>(smem);
  if (e == cudaSuccess) e = batch_round_attr<0, 4>(smem);
  if (e == cudaSuccess) e = batch_round_attr<1, 1>(smem);
  if (e == cudaSuccess) e = batch_round_attr<1, 3>(smem);
  if (e == cudaSuccess) e = batch_round_attr<1, 4>(smem);
  if (e == cudaSuccess) e = batch_round_attr<0, 3, true>(smem);
  if (e == cudaSuccess) e = batch_round_attr<0, 4, true>(smem);
  if (e == cudaSuccess) e = batch_round_attr<1, 3, true>(smem);
  if (e == cudaSuccess) e = batch_round_attr<1, 4, true>(smem);
  return e;
}

// CTAs per SM every round-kernel variant reaches with this shared memory.
cudaError_t batch_ctas_per_sm(size_t smem, int* ctas) {
  constexpr int NV = 10;
  int c[NV];
  cudaError_t e = batch_round_ctas<0, 1>(smem, &c[0]);
  if (e == cudaSuccess) e = batch_round_ctas<0, 3>(smem, &c[1]);
  if (e == cudaSuccess) e = batch_round_ctas<0, 4>(smem, &c[2]);
  if (e == cudaSuccess) e = batch_round_ctas<1, 1>(smem, &c[3]);
  if (e == cudaSuccess) e = batch_round_ctas<1, 3>(smem, &c[4]);
  if (e == cudaSuccess) e = batch_round_ctas<1, 4>(smem, &c[5]);
  if (e == cudaSuccess) e = batch_round_ctas<0, 3, true>(smem, &c[6]);
  if (e == cudaSuccess) e = batch_round_ctas<0, 4, true>(smem, &c[7]);
  if (e == cudaSuccess) e = batch_round_ctas<1, 3, true>(smem, &c[8]);
  if (e == cudaSuccess) e = batch_round_ctas<1, 4, true>(smem, &c[9]);
  if (e != cudaSuccess) return e;
  int m = c[0];
  for (int k = 1; k < NV; k++) m = c[k] < m ? c[k] : m;
  *ctas = m;
  return cudaSuccess;
}

cudaError_t launch_batch(const JobDesc* jobs, const BatchHdr* hdr, const BatchShape& sh, cudaStream_t st) {
  k_batch_sc<<<(sh.jobs_cap + 31) / 32, 32, 0, st>>>(jobs, hdr);
  k_batch_kmod<<<(sh.kmod_cap + 255) / 256, 256, 0, st>>>(jobs, hdr);
  if (sh.ks_sm_warps > 0) {
    const int smem = reserve_smem_bytes();
    cudaError_t e = allow_smem(k_batch_ks_sm<2>, smem);
    if (e != cudaSuccess) return e;
    k_batch_ks_sm<2><<<(sh.warps_cap + 1) / 2, 64, smem, st>>>(jobs, hdr);
  } else {
    k_batch_ks<<<sh.warps_cap, 32, 0, st>>>(jobs, hdr);
  }
  if (sh.rounds > 0) {
    for (int step = 0; step < sh.rounds; step++) {
      // variant v = dir * 5 + {C=1, C=3, C=4, C=3 per channel, C=4 per channel}
      if (sh.variants & (1 << 0)) k_batch_round<0, 1><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
      if (sh.variants & (1 << 1)) k_batch_round<0, 3><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
      if (sh.variants & (1 << 2)) k_batch_round<0, 4><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
      if (sh.variants & (1 << 3))
        k_batch_round<0, 3, true><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
      if (sh.variants & (1 << 4))
        k_batch_round<0, 4, true><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
      if (sh.variants & (1 << 5)) k_batch_round<1, 1><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
      if (sh.variants & (1 << 6)) k_batch_round<1, 3><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
      if (sh.variants & (1 << 7)) k_batch_round<1, 4><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
      if (sh.variants & (1 << 8))
        k_batch_round<1, 3, true><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
      if (sh.variants & (1 << 9))
        k_batch_round<1, 4, true><<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr, step);
    }
    k_batch_fixup<<<sh.grid, kRoundThreads, sh.smem, st>>>(jobs, hdr);
  }
  return cudaGetLastError();
}

// =============================================================================
// Diagnostics
// =============================================================================

__global__ void k_dbg_csin(const double* t, double* out, long long n, int variant) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = variant ? csin(t[i]) : csin_b64(t[i]);
}
__global__ void k_dbg_plcm(const double* x, const double* p, double* out, long long n, int variant) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double q = __dsub_rn(0.5, p[i]);
    out[i] = variant ? plcm_step_int(x[i], make_plcm(p[i], q)) : plcm_step(x[i], p[i], q);
  }
}
__global__ void k_dbg_lasm(const double* xymu, double* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double x = xymu[3 * i], y = xymu[3 * i + 1];
    lasm_step(x, y, __dmul_rn(kPi, xymu[3 * i + 2]));
    out[2 * i] = x;
    out[2 * i + 1] = y;
  }
}

cudaError_t launch_dbg_csin(const double* t, double* out, long long n, int variant, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_dbg_csin<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t, out, n, variant);
  return cudaGetLastError();
}
cudaError_t launch_dbg_plcm(const double* x, const double* p, double* out, long long n, int variant,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_dbg_plcm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, p, out, n, variant);
  return cudaGetLastError();
}
cudaError_t launch_dbg_lasm(const double* xymu, double* out, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_dbg_lasm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xymu, out, n);
  return cudaGetLastError();
}

}  // namespace vc
