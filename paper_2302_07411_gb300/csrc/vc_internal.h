// vc_internal.h -- types shared by the kernels (vc_kernels.cu) and the C-ABI
// layer (vc_api.cu).  Not part of the public interface.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace vc {

// An NVTX range over the host-side issue of one stage (keystream, rounds, a
// batch, a serving tick), so profilers can select kernels by stage
// (ncu --nvtx --nvtx-include "vc.keystream/").  Header-only NVTX v3: a few
// nanoseconds when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxTiles = 4096;   // tiles (row bands of the round kernels) per frame
constexpr int kMaxRowBytes = 96 * 1024;
constexpr int kRoundThreads = 256;
constexpr int kMaxSeedSlots = 1024;  // subframe seeds per tile kept in shared memory (more: computed in place)

// Frame geometry and the subframe partition (pi_i = floor(i P / n) pixels).
struct Layout {
  int H, W, C, n, rounds;
  int P;              // pixels per frame
  int N;              // bytes per frame (< 2^31)
  long long Npad;     // stride of internal per-frame buffers (multiple of 256)
  int T;              // rows per tile of the round kernels (power of two <= 32)
  int NT;             // tiles per frame = ceil(H / T)
  int SC;             // shared-memory seed slots per tile (>= the subframe starts in any tile; 0: none)
  // The diffusion of a tile runs in sub-tiles of R rows, one warp each (T / R
  // <= 8 of them per tile); a sub-tile's bytes before its first subframe start
  // stay relative to the chain value at the end of the previous sub-tile until
  // the next round (or the fix-up) reads them.
  int R, lgR;         // rows per sub-tile, a power of two: max(1, T / 8); lgR = log2(R)
  int NS;             // sub-tiles per frame = ceil(H / R)
  int ZS;             // stride of a tile row in shared memory: 32-bit pixel slots (C = 3, 4) or bytes (C = 1)
};

// Bytes of one tile row in shared memory: a 32-bit word per pixel for C = 3
// and 4, with one extra word after every 32 pixels (column o in slot
// o + o / 32, which spreads the lanes of a warp over the banks), the row
// stride even so that consecutive rows start on different banks; one byte per
// pixel for C = 1.
__host__ __device__ inline int tile_row_stride(int W, int C) {
  return C == 1 ? W : ((W + (W >> 5) + 2) & ~1);
}
__host__ __device__ inline long long tile_row_bytes(int W, int C) {
  return C == 1 ? (long long)W : 4LL * tile_row_stride(W, C);
}

// Read-only per-layout tables built on the device at init.
struct Tables {
  const int* pi;          // [n+1] first pixel of each subframe, pi[n] = P
  const uint32_t* sbits;  // [P/32 + 1] bit p set <=> pixel p starts a subframe
  const int* srank;       // [P/32 + 1] number of subframe starts before bit-word w
  const int* fixlim;      // [NS] first subframe-start byte at or after the sub-tile's first byte (or its end)
};

// Device-resident chaotic state of the n assistant PRBGs (Alg. 2).
struct Chains {
  double* st;         // PLCM: {x1, x2} per chain; 2DLASM: {x1, y1, x2, y2}
  double* par;        // PLCM: {p1, q1, p2, q2} with q = RN(1/2 - p); 2DLASM: {pm1, pm2} with pm = RN(pi mu)
  uint64_t* carry;    // [2] per chain: unconsumed bytes of the last iterate, first byte lowest
  int* carry_len;     // per chain, 0..11
};

// PRBG_m of Alg. 1 (one per stream).
struct MainPrbg {
  double s[4];        // PLCM pair {x1, p1, x2, p2}; 2DLASM single {x, y, mu, 0}; logistic pair {x1, r1, x2, r2}
  uint64_t carry[2];  // unconsumed bytes, first byte lowest
  int carry_len;
  int kind;
};

// One job of a ragged batch: nframes consecutive frames of one stream in one
// direction, with its scratch in the batch's pool.  warp_base / tile_base /
// kmod_base are the job's first index in the batch-wide work lists of the
// keystream (16 subframes per warp), round (frame x tile) and shift-table
// kernels; each list is the jobs' ranges laid end to end.
struct JobDesc {
  Layout L;
  Tables tb;
  Chains ch;
  MainPrbg* main;
  int kind, dir, nframes;
  int sine_b64;             // 2DLASM keystream: 1 = the all-binary64 sine reduction (shorter chain), 0 = integer-assisted
  const uint8_t* in;
  uint8_t* out;
  uint8_t* ks;
  long long* sc;
  int* kmod;
  uint8_t* buf[2];
  uint8_t* agg[2];
  int warp_base, tile_base, kmod_base;
  int mode;                 // 0: keystream + rounds; 1: rounds on keystream already in the ring; 2: keystream only
  int ring_cap, ring_slot0; // ks / sc / kmod frame slots: ring of ring_cap (0 = frames laid end to end)
  int pc;                   // per-channel diffusion chains (C > 1): word carries and aggregates
  int pad2;
};

// Round-kernel variants: (direction, channels, per-channel chains) -> index
// dir * 5 + {C=1: 0, C=3: 1, C=4: 2, C=3 per channel: 3, C=4 per channel: 4}.
constexpr int kBatchVariants = 10;
__host__ __device__ inline int batch_variant(int dir, int C, bool pc = false) {
  return dir * 5 + (C == 1 ? 0 : (C == 3 ? 1 : 2)) + (pc && C > 1 ? 2 : 0);
}

struct BatchHdr {
  int njobs, total_warps, total_tiles, total_kmod;
  // the jobs are ordered by variant: its tiles are [vbeg[v], vend[v])
  int vbeg[kBatchVariants], vend[kBatchVariants];
};

// Launch geometry of a batch: capacities (work beyond the header's totals
// exits at once, so one captured graph serves every batch within them);
// rounds = 0 launches the keystream phases only.
struct BatchShape {
  int jobs_cap, warps_cap, kmod_cap, rounds, grid;
  int variants;     // bit v set: a round kernel of variant v is launched
  int ks_sm_warps;  // > 0: the keystream in CTAs of this many warps that each hold a whole SM; 0: one-warp CTAs
  size_t smem;
};

}  // namespace vc

struct vc_ctx;
namespace vc {

// For a caller inside the library that is about to destroy CUDA stream `s`:
// if `s` is the stream of the context's last work, the context's internal
// keystream stream waits (on the device, the host does not block) for what
// was enqueued on `s`, and the context forgets `s` (vc_api.cu).
void ctx_release_stream(vc_ctx* c, cudaStream_t s);

// Launchers (vc_kernels.cu).  All enqueue on `st` and return the launch error.
cudaError_t launch_build_tables(const Layout& L, int* pi, uint32_t* sbits, int* srank, int* fixlim, cudaStream_t st);
cudaError_t launch_key_schedule(int kind, MainPrbg* main, Chains ch, int n, cudaStream_t st);
// cap > 0: frame f's s_c / shift table / keystream go to slot (slot0 + f) mod cap of a ring.
cudaError_t launch_frame_schedule(const Layout& L, MainPrbg* main, int nframes, long long* sc, int* kmod,
                                  cudaStream_t st, int cap = 0, int slot0 = 0);
// plcm_int: 0 binary64 pipe, 1 integer pipes, 2 integer pipes with every
// iterate sent through the exact fallback, 3 the same for odd subframes only
// (test modes of the lane-pair form).
// sm_warps > 0: CTAs of sm_warps (<= 4) warps, each holding all of an SM's shared
// memory so that no round CTA shares its SM (the chains are latency-bound and
// lose issue slots to co-resident round warps); 0: one-warp CTAs anywhere.
cudaError_t launch_keystream(int kind, const Layout& L, Tables tb, Chains ch, int nframes, uint8_t* ks,
                             int plcm_int, cudaStream_t st, int cap = 0, int slot0 = 0, int sm_warps = 0);
cudaError_t launch_keystream_thread(int kind, const Layout& L, Tables tb, Chains ch, int nframes, uint8_t* ks,
                                    int plcm_int, cudaStream_t st);
// The round kernels.  pc: per-channel diffusion chains (the alternative
// reading of Eq. 3 / Eq. 4: byte ch of a pixel chains to byte ch of the
// previous pixel, carries and aggregates one word per sub-tile) instead of one
// chain over the subframe's bytes; with C = 1 the two are the same.  The
// aggregate buffers hold NS bytes per frame (NS words with pc).  A round's
// in and out must not overlap.
cudaError_t launch_enc_round(const Layout& L, Tables tb, const uint8_t* in, long long in_stride, uint8_t* out,
                             long long out_stride, const uint8_t* ks_round, long long ks_stride, const int* kmod,
                             const uint8_t* agg_in, uint8_t* agg_out, int nframes, cudaStream_t st, bool pc = false);
cudaError_t launch_enc_fixup(const Layout& L, Tables tb, uint8_t* out, long long out_stride, const uint8_t* agg,
                             int nframes, cudaStream_t st, bool pc = false);
cudaError_t launch_dec_round(const Layout& L, Tables tb, const uint8_t* in, long long in_stride, uint8_t* out,
                             long long out_stride, const uint8_t* ks_round, long long ks_stride, const int* kmod,
                             int nframes, cudaStream_t st, bool pc = false);
// encryption round CTA (the largest of the round kernels)
size_t round_smem_bytes(const Layout& L, bool pc = false);
cudaError_t prepare_batch_kernels(size_t smem);
cudaError_t batch_ctas_per_sm(size_t smem, int* ctas);
cudaError_t launch_batch(const JobDesc* jobs, const BatchHdr* hdr, const BatchShape& sh, cudaStream_t st);

// Diagnostics: the chaotic primitives applied elementwise.
cudaError_t launch_dbg_csin(const double* t, double* out, long long n, int variant, cudaStream_t st);
cudaError_t launch_dbg_plcm(const double* x, const double* p, double* out, long long n, int variant,
                            cudaStream_t st);
cudaError_t launch_dbg_lasm(const double* xymu, double* out, long long n, cudaStream_t st);

}  // namespace vc
