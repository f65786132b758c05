// Batched step: many independent domains of uneven column and level counts
// in one launch.
//
// Work is split into items (a domain and a chunk of `blockDim.x` of its
// columns).  A persistent grid (one wave of resident blocks) takes items from
// a global atomic counter, so uneven domains balance dynamically; items of
// the domains with the most levels come first.  Optionally a flag pass first
// compacts each domain's active columns (any level the chain would change)
// into a list, and the step then runs over list entries only; columns left
// out are exactly those the step would leave unchanged, so results are
// bitwise identical with and without the list, for every block size and for
// persistent or one-item-per-block grids.  The only cross-block interaction
// is the work counter (atomicAdd); no block ever waits on another.
#pragma once

#include "casim_device.cuh"

namespace casim_dev {

constexpr int kBatchMaxBlock = 256;
constexpr int kBatchNarrowBlock = 128;
constexpr int kTile = 128;   // columns per block of the compaction pass

struct DomDesc {
  double *fld;
  long long pitch;
  const double *dz;
  double *precip;
  int ncols, nlev;
  double dzmin;    // smallest layer thickness of the domain
  long long list_off;
  long long pt_off;   // first point of the domain in a batch-wide per-point array (surrogate rates)
};

struct Item {
  int dom, chunk;
};

struct BatchArgs {
  const DomDesc *dom;
  const Item *items;   // step items (chunks of blockDim.x columns or list entries)
  int nitems;
  int *list;           // active-column indices, one segment per domain
  int *count;          // active columns per domain
  int *counter;        // work counter of the persistent grid
  unsigned *err;
  double dt;
  int compact;
  int persistent;
  const float4 *surr;   // surrogate warm-rain rates of every point of the batch (pt_off per domain), or null
  int maxlev;           // most levels of any domain (the level tables' size)
  int ndom;             // domains in the table
};

// dynamic shared memory of the batched step: the mixed step's prefetch stage
// (two levels of 16 fields per thread) and the level tables of maxlev levels
template <class M>
__host__ __device__ constexpr size_t batch_smem_bytes(int block, int maxlev) {
  return (step_staged<M, false>() ? stage_bytes<M>(block) : 0) + (size_t)maxlev * 24;
}

template <class M>
__device__ __forceinline__ bool point_needs_step(const KParams &P, const DomDesc &d, int k, int c) {
  const double *b = d.fld + (size_t)k * d.pitch + c;
  const size_t fs = (size_t)d.nlev * (size_t)d.pitch;
  Pt s;
  s.T = b[0]; s.qv = b[1 * fs]; s.qc = b[2 * fs]; s.qr = b[3 * fs];
  s.qi = b[4 * fs]; s.qs = b[5 * fs]; s.qg = b[6 * fs];
  s.p = __ldg(b + 13 * fs);
  // a non-finite value is passed on to the step, which reports it
  const unsigned h = max(max(max(hiabs(s.T), hiabs(s.qv)), max(hiabs(s.qc), hiabs(s.qr))),
                         max(max(hiabs(s.qi), hiabs(s.qs)), max(hiabs(s.qg), hiabs(s.p))));
  if (h >= 0x7ff00000u) return true;
  if constexpr (!M::kMixed) {
    double es0, qs0;
    return F64::active(P.d, s, es0, qs0);
  } else {
    W<float> w;
    float es0, qs0;
    return Mix::active(P.f, s, P.T0, w, es0, qs0);
  }
}

// Flag pass: one block per tile of kTile columns of one domain; the active
// columns of the tile are appended, in column order, to the domain's list.
template <class M>
__global__ void __launch_bounds__(kTile) k_compact(const BatchArgs b, const Item *tiles, int ntiles, const KParams P) {
  __shared__ int s_warp[kTile / 32];
  __shared__ int s_base;
  if ((int)blockIdx.x >= ntiles) return;
  const Item t = tiles[blockIdx.x];
  const DomDesc d = b.dom[t.dom];
  const int c = t.chunk * kTile + threadIdx.x;
  bool act = false;
  if (c < d.ncols)
    for (int k = d.nlev - 1; k >= 0 && !act; --k) act = point_needs_step<M>(P, d, k, c);
  const unsigned ball = __ballot_sync(0xffffffffu, act);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s_warp[wid] = __popc(ball);
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int i = 0; i < kTile / 32; ++i) {
      const int n = s_warp[i];
      s_warp[i] = tot;
      tot += n;
    }
    s_base = tot ? atomicAdd(&b.count[t.dom], tot) : 0;
  }
  __syncthreads();
  if (act) {
    const int pos = s_base + s_warp[wid] + __popc(ball & ((1u << lane) - 1u));
    if (CASIM_INDEX_OK(pos < d.ncols, b.err)) b.list[d.list_off + pos] = c;
  }
}

// kNarrow: built for blocks of at most kBatchNarrowBlock threads with the
// policy's register budget (the single-domain step's blocks per SM); else for
// blocks up to kBatchMaxBlock
template <class M, bool kNarrow = false>
__global__ void __launch_bounds__(kNarrow ? kBatchNarrowBlock : kBatchMaxBlock,
                                  kNarrow ? M::kMinBlocks : (M::kMixed ? 2 : 1))
    k_step_batch(const BatchArgs b, const KParams P) {
  extern __shared__ __align__(16) unsigned char batch_dyn[];
  __shared__ int s_item;
  const int B = blockDim.x;
  constexpr bool kStage = step_staged<M, false>();
  double *stage = kStage ? reinterpret_cast<double *>(batch_dyn) : nullptr;
  double *s_dz = reinterpret_cast<double *>(batch_dyn + (kStage ? stage_bytes<M>(B) : 0));
  double *s_dzdt = s_dz + b.maxlev;
  float *s_dtdz_f = reinterpret_cast<float *>(s_dzdt + b.maxlev), *s_dzdt_f = s_dtdz_f + b.maxlev;
  const LevelTab lt{s_dz, s_dzdt, s_dtdz_f, s_dzdt_f};
  const int tid = threadIdx.x;
  unsigned eflag = 0;
  int prev_dom = -1;
  for (int iter = 0;; ++iter) {
    int it;
    if (b.persistent) {
      if (tid == 0) s_item = atomicAdd(b.counter, 1);
      __syncthreads();
      it = s_item;
    } else {
      it = iter == 0 ? (int)blockIdx.x : b.nitems;
    }
    if (it >= b.nitems) break;
    const Item item = b.items[it];
    if (!CASIM_INDEX_OK(item.dom >= 0 && item.dom < b.ndom, b.err)) break;
    const DomDesc d = b.dom[item.dom];
    const int n = b.compact ? b.count[item.dom] : d.ncols;
    if (item.chunk * B < n) {
      if (item.dom != prev_dom) {
        for (int k = tid; k < d.nlev; k += B) level_tab(s_dz, s_dzdt, s_dtdz_f, s_dzdt_f, k, d.dz[k], b.dt);
        __syncthreads();
        prev_dom = item.dom;
      }
      bool fast = true;
#pragma unroll
      for (int x = 1; x < 5; ++x) fast &= ((P.vmax[x] * b.dt) / d.dzmin) / P.c_max <= 1.0;
      const int idx = item.chunk * B + tid;
      if (idx < n) {
        const int c = b.compact && CASIM_INDEX_OK(idx < d.ncols, b.err) ? b.list[d.list_off + idx] : idx;
        KArgs a;
        a.fld = d.fld;
        a.pitch = d.pitch;
        a.dz = d.dz;
        a.precip = d.precip;
        a.err = b.err;
        a.ncols = d.ncols;
        a.nlev = d.nlev;
        a.dt = b.dt;
        a.surr = b.surr ? b.surr + d.pt_off : nullptr;
        a.stats = nullptr;
        eflag |= run_column<M, false, kStage>(a, P, lt, fast, c, nullptr, kStage ? stage + tid : nullptr, B);
      }
    }
    // shared memory (item, dz) is reused by the next item; with one item per
    // block there is none, and the warps leave as they finish
    if (b.persistent) __syncthreads();
  }
  if (eflag) atomicOr(b.err, eflag);
}

}  // namespace casim_dev
