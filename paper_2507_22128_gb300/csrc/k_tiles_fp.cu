// a5 + a6 (Eq. 2), FP32 w-stacked: degrid, residual and grid of one uv
// partition with register-resident kernel footprints.
//
// The medium and large workloads are dense: tens of samples of one w-plane
// block fall on each uv cell, so many samples share the exact 8 x 8 x 8 tap
// footprint (same first tap in u, v and w).  At partition time the entries
// of every work item (one 16 x 16 tile of one w-plane block) are reordered by
// their first tap and cut into chunks: runs of entries with one footprint, at
// most the job's chunk limit (64 by default, up to 256).  Per call,
// k_gather_y writes every entry's weighted visibility {w re v, w im v, w} in
// that order, so the gridder reads a chunk as contiguous runs of 512 bytes.
// The kernel gives each chunk to one warp (warps claim an item's chunks from
// a shared-memory queue), which works through it in batches of up to 32
// entries, fetching the next batch by cp.async while it works on the
// current one, and
//   * reads the footprint's 512 model cells from the staged tile once per
//     chunk into registers (lane: v row = lane & 7, planes lane >> 3 and that
//     + 4, all 8 u taps: 16 complex cells, held as FP32 pairs of adjacent u
//     taps),
//   * per pair of samples forms the 2 x 24 kernel weights (one
//     exponential-of-semicircle evaluation per weight, spread over the
//     lanes), degrids both with packed FP32x2 FMAs, reduces them with a
//     transposed butterfly (10 shuffles for the pair), forms the weighted
//     residuals and spreads them into 16 complex accumulators per lane,
//   * adds its accumulators into the shared-memory grid tile once per chunk,
//     with plain read-modify-writes under a per-CTA lock (warps of one item
//     may share cells).
// The model tile (8 planes x 23 x 24 complex cells, the tile plus the kernel
// halo) arrives by one TMA tensor load per item, completion tracked by an
// mbarrier; the item's grid tile leaves by one TMA bulk reduce-add into the
// partition's residual planes (element-wise atomic in L2), replacing
// per-cell global atomics.  Tensor maps cover this GPU's own memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "rix_internal.cuh"

namespace rix {
namespace {

constexpr int kT = 16;                        // tile side (cells)
constexpr int kSide = kT + kW - 1;            // staged side in u: tile + kernel halo
constexpr int kRow = 24;                      // staged row in v (complex cells): TMA box of 48 floats = 192 B
constexpr int kPlaneC = kSide * kRow;         // complex cells per staged plane (552 == 8 mod 16)
constexpr int kTileFloats = kW * kPlaneC * 2; // 8 planes
constexpr int kTileBytes = kTileFloats * 4;   // 35,328 B (a multiple of 128)
constexpr int kChunkMax = 32;                 // entries per batch (a warp's staging slot)
constexpr int kChunkLimitMax = 256;           // most entries per chunk (the job's chunk limit)
constexpr int kItemMax = 2048;                // entries per work item (the partition's item split)
constexpr int kFpThreads = 256;
constexpr int kFpWarps = kFpThreads / 32;
constexpr uint32_t kWaitPolls = 1u << 24;     // bounded mbarrier wait
constexpr uint32_t kLockPolls = 1u << 22;     // bounded wait for the grid tile's flush lock
static_assert(kTileBytes % 128 == 0, "tile alignment");

// ------------------------------------------------------ partition time -----
// Per work item: reorder its entries (at most 2048) by first tap, stably
// (key = tap << 11 | position), the geometry records in place and the sample
// indices (read from `samples`, in the geometry's current order: the sorted
// order at partition time, the gridder order when the chunks are rebuilt)
// into gsamples (which may be `samples`), and flag the entries
// that start a chunk (the first of a run of one tap, and every limit-th
// after; limit <= 32, the job's tuning).
template <typename R>
__global__ void __launch_bounds__(256) k_item_order(const uint32_t* __restrict__ items, int64_t n_items,
                                                    const uint32_t* samples, EntryGeom<R>* geom,
                                                    uint32_t* gsamples, uint32_t* __restrict__ cflag,
                                                    int limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EntryGeom<R>* sg = reinterpret_cast<EntryGeom<R>*>(smem_raw);
  uint32_t* sk = reinterpret_cast<uint32_t*>(sg + kItemMax);
  uint32_t* ss = sk + kItemMax;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const uint32_t e0 = items[item];
    const int cnt = (int)(items[item + 1] - e0);
    int p2 = 2;
    while (p2 < cnt) p2 <<= 1;
    for (int r = threadIdx.x; r < p2; r += blockDim.x) {
      if (r < cnt) {
        const EntryGeom<R> g = geom[e0 + r];
        sg[r] = g;
        ss[r] = samples[e0 + r];
        sk[r] = ((g.ouv & 0xffffu) << 11) | (uint32_t)r;
      } else {
        sk[r] = 0xffffffffu;
      }
    }
    __syncthreads();
    // bitonic sort of sk[0, p2) ascending
    for (int k = 2; k <= p2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < p2; i += blockDim.x) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const uint32_t x = sk[i], y = sk[ixj];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              sk[i] = y;
              sk[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
      const uint32_t key = sk[r];
      const int src = (int)(key & 2047u);
      gsamples[e0 + r] = ss[src];
      geom[e0 + r] = sg[src];
      // position of the first entry with this tap (lower bound of tap << 11)
      const uint32_t lo_key = key & ~2047u;
      int lo = 0, hi = r;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sk[mid] < lo_key) lo = mid + 1;
        else hi = mid;
      }
      cflag[e0 + r] = ((r - lo) % limit) == 0 ? 1u : 0u;
    }
    __syncthreads();
  }
}

// chunks[cidx[e]] = e for the chunk-start entries; item_chunk[i] =
// cidx[items[i]] (every item starts a chunk); sentinels at the ends
__global__ void k_chunk_lists(const uint32_t* __restrict__ cflag, const uint32_t* __restrict__ cidx, int64_t n_ent,
                              const uint32_t* __restrict__ items, int64_t n_items, const uint32_t* __restrict__ total,
                              uint32_t* __restrict__ chunks, uint32_t* __restrict__ item_chunk) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_ent; e += stride)
    if (cflag[e]) chunks[cidx[e]] = (uint32_t)e;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_items; i += stride)
    item_chunk[i] = cidx[items[i]];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    chunks[*total] = (uint32_t)n_ent;
    item_chunk[n_items] = *total;
  }
}

// ------------------------------------------------------- the PSF's grid ----
// The PSF (H of Eq. 4-7) is the dirty image of unit visibilities on the 2N x
// 2N field, gridded on that field's own oversampled grid (side 4N).  Its
// entries are the partition's, sorted once per job by their 16 x 16 tile of
// the PSF grid (tiles counted from the partition's PSF window) and w-plane
// block, cut into work items and chunks as on the image grid.
struct PsfArgs {
  const uint32_t* keys;      // image-grid sort keys (the plane block)
  const uint32_t* samples;   // sample index per entry (image gridder order)
  const double* uvw;
  const double* inv_lambda;
  int nchan;
  double scale, half;        // PSF grid coordinate x = u_lambda * scale + half
  int nw, ww;
  double w_min, dw;
  int bt_img, bt, bw;        // key bits per tile coordinate (image grid, PSF window), plane bits
  int win_lo, win_n;         // the partition's PSF window [win_lo, win_lo + win_n)^2
  int64_t e_begin, n;        // the partition's entries
  int* status;
};

// Per entry (local index i = entry - e_begin): the geometry record on the PSF
// grid {du, dv, dw, first tap's offsets in its PSF tile}, the PSF key (plane
// block, tile row, tile column) and i itself (the sort's payload); FP64
// coordinates as k_entry_geom.
__global__ void k_psf_geom(PsfArgs a, float4* __restrict__ geom, uint32_t* __restrict__ pkey,
                           uint32_t* __restrict__ idx) {
  const uint32_t pmask = (1u << a.bw) - 1u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = a.e_begin + i;
    const uint32_t p0 = (a.keys[e] >> (2 * a.bt_img)) & pmask;
    const uint32_t s = a.samples[e];
    const int64_t row = s / (uint32_t)a.nchan;
    const int ch = (int)(s - row * a.nchan);
    const double sc = a.inv_lambda[ch];
    const double ul = __dmul_rn(a.uvw[row * 3 + 0], sc);
    const double vl = __dmul_rn(a.uvw[row * 3 + 1], sc);
    const double x = __dadd_rn(__dmul_rn(ul, a.scale), a.half);
    const double y = __dadd_rn(__dmul_rn(vl, a.scale), a.half);
    const double xs = __dadd_rn(x, -0.5 * kW), ys = __dadd_rn(y, -0.5 * kW);
    const double cx = ceil(xs), cy = ceil(ys);
    int ju = (int)cx - a.win_lo, jv = (int)cy - a.win_lo;
    float dw = 0.f;
    if (a.nw > 0) {
      const double wl = __dmul_rn(a.uvw[row * 3 + 2], sc);
      const double tw = __ddiv_rn(__dadd_rn(wl, -a.w_min), a.dw);
      const double pc = fmin(fmax(ceil(tw), 0.0), (double)(a.nw - a.ww));
      dw = (float)__dadd_rn(pc, -tw);
    }
    // the window holds every footprint of the partition by construction; an
    // entry outside it is flagged (RIX_EINTERNAL) and kept in range
    if (ju < 0 || jv < 0 || ju > a.win_n - kW || jv > a.win_n - kW) {
      atomicCAS(a.status, 0, RIX_EINTERNAL);
      ju = min(max(ju, 0), a.win_n - kW);
      jv = min(max(jv, 0), a.win_n - kW);
    }
    const uint32_t ouv = (uint32_t)(ju & (kT - 1)) | ((uint32_t)(jv & (kT - 1)) << 8);
    geom[i] = make_float4((float)__dadd_rn(cx, -xs), (float)__dadd_rn(cy, -ys), dw, __uint_as_float(ouv));
    pkey[i] = (p0 << (2 * a.bt)) | ((uint32_t)(jv / kT) << a.bt) | (uint32_t)(ju / kT);
    idx[i] = (uint32_t)i;
  }
}

// After the stable sort of the PSF keys (sk, with the local entry indices
// sv): f[i] = 1 where a run of equal keys starts.
__global__ void k_psf_runs(const uint32_t* __restrict__ sk, int64_t n, uint32_t* __restrict__ f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    f[i] = (i == 0 || sk[i] != sk[i - 1]) ? 1u : 0u;
}

// first entry of every run (ex: exclusive scan of the run flags)
__global__ void k_psf_run_starts(const uint32_t* __restrict__ f, const uint32_t* __restrict__ ex, int64_t n,
                                 uint32_t* __restrict__ starts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (f[i]) starts[ex[i]] = (uint32_t)i;
}

// The geometry and weight of every entry in key order, and the entries that
// start a work item (the first of a run, and every kItemMax-th after it).
__global__ void k_psf_gather(const uint32_t* __restrict__ sv, const float4* __restrict__ geom_in,
                             const uint32_t* __restrict__ samples, const float* __restrict__ weight, int64_t e_begin,
                             const uint32_t* __restrict__ f, const uint32_t* __restrict__ ex,
                             const uint32_t* __restrict__ starts, int64_t n, float4* __restrict__ geom,
                             float* __restrict__ w, uint32_t* __restrict__ iflag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t src = sv[i];
    geom[i] = geom_in[src];
    w[i] = weight ? weight[samples[e_begin + src]] : 1.0f;
    const uint32_t run = ex[i] + f[i] - 1u;
    iflag[i] = (((uint32_t)i - starts[run]) % (uint32_t)kItemMax) == 0u ? 1u : 0u;
  }
}

// work-item start offsets (iex: exclusive scan of the item flags; sentinel n)
__global__ void k_psf_items(const uint32_t* __restrict__ iflag, const uint32_t* __restrict__ iex, int64_t n,
                            const uint32_t* __restrict__ n_items, uint32_t* __restrict__ items) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (iflag[i]) items[iex[i]] = (uint32_t)i;
  if (blockIdx.x == 0 && threadIdx.x == 0) items[*n_items] = (uint32_t)n;
}

// Per work item (one PSF tile of one w-plane block, at most kItemMax entries;
// *n_items of them): the entries reordered stably by first tap, their unit
// visibilities {w, 0, w, 0} written in that order, and the entries that
// start a chunk (a new first tap, and every limit-th after) flagged.
__global__ void __launch_bounds__(256) k_psf_order(const uint32_t* __restrict__ items,
                                                   const uint32_t* __restrict__ n_items, const float* __restrict__ w,
                                                   float4* geom, float4* __restrict__ ysamp,
                                                   uint32_t* __restrict__ cflag, int limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* sg = reinterpret_cast<float4*>(smem_raw);
  uint32_t* sk = reinterpret_cast<uint32_t*>(sg + kItemMax);
  float* sw = reinterpret_cast<float*>(sk + kItemMax);
  const int64_t ni = *n_items;
  for (int64_t it = blockIdx.x; it < ni; it += gridDim.x) {
    const uint32_t e0 = items[it];
    const int cnt = (int)(items[it + 1] - e0);
    int p2 = 2;
    while (p2 < cnt) p2 <<= 1;
    for (int r = threadIdx.x; r < p2; r += blockDim.x) {
      if (r < cnt) {
        const float4 g = geom[e0 + r];
        sg[r] = g;
        sw[r] = w[e0 + r];
        const uint32_t ouv = __float_as_uint(g.w);
        sk[r] = ((((ouv >> 8) << 4) | (ouv & 0xffu)) << 11) | (uint32_t)r;   // 8-bit tap, position
      } else {
        sk[r] = 0xffffffffu;
      }
    }
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < p2; i += blockDim.x) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const uint32_t x = sk[i], y = sk[ixj];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              sk[i] = y;
              sk[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
      const uint32_t key = sk[r];
      const int src = (int)(key & 2047u);
      geom[e0 + r] = sg[src];
      ysamp[e0 + r] = make_float4(sw[src], 0.f, sw[src], 0.f);
      const uint32_t lo_key = key & ~2047u;
      int lo = 0, hi = r;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sk[mid] < lo_key) lo = mid + 1;
        else hi = mid;
      }
      cflag[e0 + r] = ((r - lo) % limit) == 0 ? 1u : 0u;
    }
    __syncthreads();
  }
}

// chunk lists of the PSF's entries: chunks[cidx[e]] = e at the flagged
// entries, item_chunk[i] = cidx[items[i]]; sentinels at the ends
__global__ void k_psf_lists(const uint32_t* __restrict__ cflag, const uint32_t* __restrict__ cidx, int64_t n,
                            const uint32_t* __restrict__ items, const uint32_t* __restrict__ n_items,
                            const uint32_t* __restrict__ n_chunks, uint32_t* __restrict__ chunks,
                            uint32_t* __restrict__ item_chunk) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t ni = *n_items;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride)
    if (cflag[e]) chunks[cidx[e]] = (uint32_t)e;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += stride)
    item_chunk[i] = cidx[items[i]];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    chunks[*n_chunks] = (uint32_t)n;
    item_chunk[ni] = *n_chunks;
  }
}

// ------------------------------------------------------------- PTX glue ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// 3D tiled TMA load (coordinates fastest first) completing on `bar`
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// 3D tiled TMA reduce-add of shared memory into global memory
__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap* map, int x, int y, int z, uint32_t src) {
  asm volatile("cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   (uint64_t)map),
               "r"(x), "r"(y), "r"(z), "r"(src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

struct FpArgs {
  const uint32_t* keys;
  const uint32_t* items;       // entry offset of each work item (+ sentinel)
  const uint32_t* item_chunk;  // first chunk of each work item (+ sentinel)
  const uint32_t* chunks;      // entry offset of each chunk (+ sentinel)
  const float4* geom;          // EntryGeom<float> per entry, gridder order
  const float4* ysamp;         // per entry: {w re v, w im v, w, 0}, gridder order
  int64_t item_begin, item_count;
  const uint32_t* dev_items;   // grid mode: null, or the number of work items in device memory (item_count bounds it)
  int bt, bw, win_lo;
  int* status;                 // the job's status word
};

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGroup = 2;                     // samples degridded, reduced and gridded together
constexpr int kCbMax = 1024;                  // chunk bounds of an item staged in shared memory

// Exponential-of-semicircle weight of tap i (see es_weight) from the
// hardware approximations: sqrt.approx and exp(x) = 2^(x log2 e) by
// ex2.approx (relative errors near 2^-22, far below the FP32 operator's
// 1e-5 bound).
__device__ __forceinline__ float es_weight_fast(float d, int i) {
  const float z = fmaf(d + (float)i, 2.0f / kW, -1.0f);
  const float t = fmaxf(fmaf(-z, z, 1.0f), 0.0f);
  float r, e;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
  const float x = (float)(kBeta * 1.4426950408889634) * (r - 1.0f);
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(x));
  return e;
}

// Packed FP32 pairs held as 64-bit register pairs (lo = first element) for
// the f32x2 FMA: d = a * b + c element-wise.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x ffma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2x pack2(float lo, float hi) {
  f2x d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ float2 unpack2(f2x v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ float hsum2(f2x v) {
  const float2 r = unpack2(v);
  return r.x + r.y;
}

// keep-or-send exchange of one butterfly stage: the lane keeps the half its
// lane bit selects and adds the partner's copy of the same sample
__device__ __forceinline__ float2 bfly(bool hi, float2 lo_v, float2 hi_v, int mask) {
  const float2 keep = hi ? hi_v : lo_v;
  const float2 send = hi ? lo_v : hi_v;
  return make_float2(keep.x + __shfl_xor_sync(kFull, send.x, mask), keep.y + __shfl_xor_sync(kFull, send.y, mask));
}

// 16-byte asynchronous global -> shared copy (cp.async, cached at L2 only)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// per warp: two chunk slots ({du, dv, dw, tap} and {w re v, w im v, w, 0} of
// up to 32 entries) and the weights of one group of samples
struct WarpScratch {
  float4 g[2][kChunkMax];
  float4 y[2][kChunkMax];
  float w[kGroup * 24];
};

// Several partitions (of one or more jobs) in one launch: per pair its
// arguments and its two tensor maps (model planes, residual planes; 64-byte
// aligned device array), and the first global work item of every pair
// (n + 1 values: item_start[n] = the total).
struct FpBatch {
  const FpArgs* descs;
  const CUtensorMap* maps;
  const int64_t* item_start;
  int n;
};

template <int MODE, bool BATCH>
__global__ void __launch_bounds__(kFpThreads, 2)
    k_tiles_fp(FpArgs a0, const __grid_constant__ CUtensorMap tm_model0, const __grid_constant__ CUtensorMap tm_out0,
               FpBatch bt) {
  constexpr bool kModel = (MODE == kResid);
  __shared__ FpArgs sa;   // the arguments of the pair the CTA works on
  if (!BATCH && threadIdx.x == 0) sa = a0;
  const FpArgs& a = sa;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* grid = reinterpret_cast<float*>(base);
  const float2* model = reinterpret_cast<const float2*>(base + kTileBytes);
  unsigned char* tail = base + (kModel ? 2 : 1) * kTileBytes;
  WarpScratch* scratch = reinterpret_cast<WarpScratch*>(tail);
  uint32_t* cb = reinterpret_cast<uint32_t*>(scratch + kFpWarps);   // chunk bounds of the item
  uint32_t* queue = cb + kCbMax;                                     // next chunk to claim
  uint32_t* lock = queue + 1;                                        // the grid tile's flush lock
  uint64_t* bar = reinterpret_cast<uint64_t*>(queue + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vrow = lane & 7, pa = lane >> 3;         // this lane's v row and planes pa, pa + 4
  const int mine = (lane >> 4) & 1;                  // the group sample whose degrid sum this lane ends with
  const bool b4 = (lane >> 4) & 1;
  const uint32_t bar_a = smem_u32(bar);
  if (threadIdx.x == 0) *lock = 0u;
  if (kModel && threadIdx.x == 0) {
    mbar_init(bar_a, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  WarpScratch& ws = scratch[warp];
  float* wg = ws.w;

  int64_t total = BATCH ? bt.item_start[bt.n] : a0.item_count;
  if constexpr (MODE == kGrid && !BATCH) {
    if (a0.dev_items) total = min(total, (int64_t)*a0.dev_items);
  }
  int cur = -1;
  for (int64_t it = blockIdx.x; it < total; it += gridDim.x) {
    int64_t item;
    const CUtensorMap* tm_model;
    const CUtensorMap* tm_out;
    if constexpr (BATCH) {
      // the pair of global item `it`: the last i with item_start[i] <= it
      int lo = 0, hi = bt.n - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bt.item_start[mid] <= it) lo = mid;
        else hi = mid - 1;
      }
      if (lo != cur) {
        __syncthreads();
        if (threadIdx.x == 0) sa = bt.descs[lo];
        __syncthreads();
        cur = lo;
      }
      item = a.item_begin + (it - bt.item_start[lo]);
      tm_model = bt.maps + 2 * lo;
      tm_out = bt.maps + 2 * lo + 1;
    } else {
      item = a0.item_begin + it;
      tm_model = &tm_model0;
      tm_out = &tm_out0;
    }
    const uint32_t tmask = (1u << a.bt) - 1u;
    const uint32_t e0 = a.items[item];
    const uint32_t key = a.keys[e0];
    const int tx = (int)(key & tmask), ty = (int)((key >> a.bt) & tmask);
    const int p0 = (int)((key >> (2 * a.bt)) & ((1u << a.bw) - 1u));
    const int u0 = tx * kT - a.win_lo, v0 = ty * kT - a.win_lo;   // >= 0: the window is tile-aligned
    if (kModel && threadIdx.x == 0) {
      mbar_expect_tx(bar_a, kTileBytes);
      tma_load_3d(smem_u32(model), tm_model, 2 * v0, u0, p0, bar_a);
    }
    const uint32_t c0 = a.item_chunk[item];
    const int nch = (int)(a.item_chunk[item + 1] - c0);
    float4* g4 = reinterpret_cast<float4*>(grid);
    for (int i = threadIdx.x; i < kTileFloats / 4; i += kFpThreads) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = threadIdx.x; i <= nch && i < kCbMax; i += kFpThreads) cb[i] = a.chunks[c0 + i];
    if (threadIdx.x == 0) *queue = 0u;
    if (kModel) {
      // one thread polls (bounded) while the others wait at the barrier,
      // leaving the issue slots to the SM's other CTA
      bool ok = true;
      if (threadIdx.x == 0) {
        ok = false;
        for (uint32_t k = 0; k < kWaitPolls && !ok; ++k) ok = mbar_try_wait(bar_a, phase);
      }
      phase ^= 1u;
      if (!__syncthreads_and(ok)) {
        // the tile never arrived: report, give the copy a last bounded
        // chance to land (it targets this CTA's shared memory), and stop
        if (threadIdx.x == 0) {
          atomicCAS(a.status, 0, RIX_ETIMEOUT);
          for (uint32_t k = 0; k < kWaitPolls && !mbar_try_wait(bar_a, phase ^ 1u); ++k) {
          }
        }
        return;
      }
    } else {
      __syncthreads();
    }

    // chunk bound i of the item (staged, or read from global past kCbMax)
    auto bound = [&](int i) -> uint32_t { return i < kCbMax ? cb[i] : a.chunks[c0 + i]; };
    // claim the next chunk of the item for this warp
    auto claim = [&]() -> int {
      int k = 0;
      if (lane == 0) k = (int)atomicAdd(queue, 1u);
      return __shfl_sync(kFull, k, 0);
    };
    // start the copies of the nb (<= 32) entries from eb into slot `sl`;
    // slot entries past nb are zero (zero weight and data)
    auto fetch = [&](uint32_t eb, int nb, int sl) {
      if (lane < nb) {
        cp_async16(&ws.g[sl][lane], a.geom + eb + lane);
        cp_async16(&ws.y[sl][lane], a.ysamp + eb + lane);
      } else {
        ws.g[sl][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        ws.y[sl][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };

    // A chunk (entries with one footprint, at most the job's chunk limit)
    // is worked through in batches of up to 32 entries: its model cells are
    // read and its accumulators flushed once per chunk, and the next batch
    // (the rest of this chunk, else the first batch of the next claimed
    // chunk) is prefetched while the current one is processed.
    int k = claim();
    int sl = 0;
    uint32_t pos = 0, end = 0;   // the current batch's first entry, the chunk's end
    if (k < nch) {
      pos = bound(k);
      end = bound(k + 1);
      fetch(pos, (int)min(end - pos, 32u), sl);
    }
    while (k < nch) {
      f2x mar[4], mai[4], mbr[4], mbi[4];   // model cells, pairs of adjacent u taps (re, im separately)
      f2x aar[4], aai[4], abr[4], abi[4];   // accumulators, the same layout
#pragma unroll
      for (int t = 0; t < 4; ++t) aar[t] = aai[t] = abr[t] = abi[t] = 0ull;
      int k2 = k;
      uint32_t npos = pos, nend = end;
      int cell = 0;
      bool first = true, more = true;
      while (more) {
        const int nb = (int)min(end - pos, 32u);
        // the next batch: the rest of this chunk, else the next chunk's first
        npos = pos + (uint32_t)nb;
        more = npos < end;
        bool next = more;
        if (!more) {
          k2 = claim();
          if (k2 < nch) {
            npos = bound(k2);
            nend = bound(k2 + 1);
            next = true;
          }
        }
        if (next) {
          fetch(npos, (int)min(nend - npos, 32u), sl ^ 1);
          asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
          asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        const float4* sd = ws.g[sl];
        const float4* sy = ws.y[sl];
        if (first) {
          first = false;
          const uint32_t ouv = __float_as_uint(sd[0].w);
          cell = (int)(ouv & 0xffu) * kRow + (int)(ouv >> 8) + vrow;   // complex cell in a plane
          if (kModel) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const float2 x0 = model[pa * kPlaneC + cell + (2 * t) * kRow];
              const float2 x1 = model[pa * kPlaneC + cell + (2 * t + 1) * kRow];
              const float2 y0 = model[(pa + 4) * kPlaneC + cell + (2 * t) * kRow];
              const float2 y1 = model[(pa + 4) * kPlaneC + cell + (2 * t + 1) * kRow];
              mar[t] = pack2(x0.x, x1.x);
              mai[t] = pack2(x0.y, x1.y);
              mbr[t] = pack2(y0.x, y1.x);
              mbi[t] = pack2(y0.y, y1.y);
            }
          }
        }
        for (int j0 = 0; j0 < nb; j0 += kGroup) {
          // ---- the group's kGroup x 24 kernel weights over the warp's lanes:
          // entry e of sample e / 24, tap e % 24 (0-7 u, 8-15 v, 16-23 w)
#pragma unroll
          for (int r = 0; r < (kGroup * 24 + 31) / 32; ++r) {
            const int e = lane + 32 * r;
            if (e >= kGroup * 24) break;
            const int kk = e / 24, tap = e - 24 * (e / 24);
            const float* dk = reinterpret_cast<const float*>(&sd[j0 + kk]);
            wg[e] = es_weight_fast(dk[tap >> 3], tap & 7);
          }
          __syncwarp();
          // per sample: the lane's v-row times w-plane weights (fa: plane pa,
          // fb: plane pa + 4)
          float fa[kGroup], fb[kGroup];
#pragma unroll
          for (int kk = 0; kk < kGroup; ++kk) {
            const float wv = wg[kk * 24 + 8 + vrow];
            fa[kk] = wv * wg[kk * 24 + 16 + pa];
            fb[kk] = wv * wg[kk * 24 + 20 + pa];
          }
          float y0 = 0.f, y1 = 0.f;   // w (v - model) of sample `mine`
          if (kModel) {
            // ---- degrid partials of the 4 samples over this lane's 16 cells
            float2 part[kGroup];
#pragma unroll
            for (int kk = 0; kk < kGroup; ++kk) {
              const ulonglong2 wlo = *reinterpret_cast<const ulonglong2*>(wg + kk * 24);
              const ulonglong2 whi = *reinterpret_cast<const ulonglong2*>(wg + kk * 24 + 4);
              const f2x wu[4] = {wlo.x, wlo.y, whi.x, whi.y};
              f2x sar = 0ull, sai = 0ull, sbr = 0ull, sbi = 0ull;
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                sar = ffma2(wu[t], mar[t], sar);
                sai = ffma2(wu[t], mai[t], sai);
                sbr = ffma2(wu[t], mbr[t], sbr);
                sbi = ffma2(wu[t], mbi[t], sbi);
              }
              part[kk] = make_float2(fmaf(fa[kk], hsum2(sar), fb[kk] * hsum2(sbr)),
                                     fmaf(fa[kk], hsum2(sai), fb[kk] * hsum2(sbi)));
            }
            // ---- transposed butterfly: the first stage exchanges half of the
            // pair, so the lane ends with the sum over all 32 lanes of sample
            // `mine` after 10 shuffles for the 2 samples
            float2 tot = bfly(b4, part[0], part[1], 16);
            tot.x += __shfl_xor_sync(kFull, tot.x, 8);
            tot.y += __shfl_xor_sync(kFull, tot.y, 8);
            tot.x += __shfl_xor_sync(kFull, tot.x, 4);
            tot.y += __shfl_xor_sync(kFull, tot.y, 4);
            tot.x += __shfl_xor_sync(kFull, tot.x, 2);
            tot.y += __shfl_xor_sync(kFull, tot.y, 2);
            tot.x += __shfl_xor_sync(kFull, tot.x, 1);
            tot.y += __shfl_xor_sync(kFull, tot.y, 1);
            const float4 ym = sy[j0 + mine];
            y0 = fmaf(-ym.z, tot.x, ym.x);
            y1 = fmaf(-ym.z, tot.y, ym.y);
          }
          // ---- grid the group's samples into the accumulators
#pragma unroll
          for (int kk = 0; kk < kGroup; ++kk) {
            const float fak = fa[kk], fbk = fb[kk];
            float yrk, yik;
            if (kModel) {
              yrk = __shfl_sync(kFull, y0, 16 * kk);
              yik = __shfl_sync(kFull, y1, 16 * kk);
            } else {
              const float4 yk = sy[j0 + kk];
              yrk = yk.x;
              yik = yk.y;
            }
            const ulonglong2 wlo = *reinterpret_cast<const ulonglong2*>(wg + kk * 24);
            const ulonglong2 whi = *reinterpret_cast<const ulonglong2*>(wg + kk * 24 + 4);
            const f2x wu[4] = {wlo.x, wlo.y, whi.x, whi.y};
            const float ar = yrk * fak, ai = yik * fak, br = yrk * fbk, bi = yik * fbk;
            const f2x car = pack2(ar, ar), cai = pack2(ai, ai), cbr = pack2(br, br), cbi = pack2(bi, bi);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              aar[t] = ffma2(car, wu[t], aar[t]);
              aai[t] = ffma2(cai, wu[t], aai[t]);
              abr[t] = ffma2(cbr, wu[t], abr[t]);
              abi[t] = ffma2(cbi, wu[t], abi[t]);
            }
          }
          __syncwarp();   // the group's weights are read before the next group overwrites them
        }
        __syncwarp();   // the slot is read before its next fetch
        sl ^= 1;
        if (more) pos = npos;
      }
      // add the chunk's accumulators into the item's grid tile: plain
      // read-modify-writes under the CTA's flush lock (the chunks of one
      // item overlap; with shared-memory float atomics instead, a launch of
      // the medium workload took 0.19 / 0.27 ms longer); a lock that stays
      // taken (impossible: every holder releases it after 16 loads and
      // stores) is reported and the flush goes ahead without it
      float* ga = grid + 2 * (pa * kPlaneC + cell);
      float* gb = grid + 2 * ((pa + 4) * kPlaneC + cell);
      bool held = false;
      if (lane == 0) {
        for (uint32_t n = 0; n < kLockPolls && !held; ++n) {
          held = atomicCAS(lock, 0u, 1u) == 0u;
          if (!held) __nanosleep(32);
        }
        if (!held) atomicCAS(a.status, 0, RIX_ETIMEOUT);
        __threadfence_block();
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float2 ar = unpack2(aar[t]), ai = unpack2(aai[t]), br = unpack2(abr[t]), bi = unpack2(abi[t]);
        float2* qa0 = reinterpret_cast<float2*>(ga + 2 * (2 * t) * kRow);
        float2* qa1 = reinterpret_cast<float2*>(ga + 2 * (2 * t + 1) * kRow);
        float2* qb0 = reinterpret_cast<float2*>(gb + 2 * (2 * t) * kRow);
        float2* qb1 = reinterpret_cast<float2*>(gb + 2 * (2 * t + 1) * kRow);
        float2 c0 = *qa0, c1 = *qa1, c2 = *qb0, c3 = *qb1;
        c0.x += ar.x; c0.y += ai.x;
        c1.x += ar.y; c1.y += ai.y;
        c2.x += br.x; c2.y += bi.x;
        c3.x += br.y; c3.y += bi.y;
        *qa0 = c0;
        *qa1 = c1;
        *qb0 = c2;
        *qb1 = c3;
      }
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        if (held) atomicExch(lock, 0u);
      }
      k = k2;
      pos = npos;
      end = nend;
    }
    // the grid tile's shared-memory writes become visible to the TMA unit,
    // then one thread adds the tile into the residual planes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      tma_reduce_add_3d(tm_out, 2 * v0, u0, p0, smem_u32(grid));
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// per entry of [e_begin, e_begin + n): ysamp = {w re v, w im v, w, 0} of its
// sample (gridder order)
__global__ void k_gather_y(const uint32_t* __restrict__ samples, const float2* __restrict__ vis,
                           const float* __restrict__ weight, int64_t e_begin, int64_t n,
                           float4* __restrict__ ysamp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = e_begin + i;
    const uint32_t s = samples[e];
    const float2 v = vis[s];
    const float w = weight ? weight[s] : 1.0f;
    ysamp[e] = make_float4(w * v.x, w * v.y, w, 0.f);
  }
}

// ------------------------------------------------------------------ host ----
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of complex planes [nplanes][S][S] seen as FP32 [nplanes][S][2S],
// box 8 planes x 23 rows x 48 floats (one staged tile).
int plane_map(CUtensorMap* map, const void* planes, int S, int nplanes) {
  auto fn = encode_fn();
  if (!fn) return set_error(RIX_ECUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[3] = {(cuuint64_t)2 * S, (cuuint64_t)S, (cuuint64_t)nplanes};
  const cuuint64_t strides[2] = {(cuuint64_t)2 * S * 4, (cuuint64_t)2 * S * 4 * S};
  const cuuint32_t box[3] = {2 * kRow, kSide, kW};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(planes), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(RIX_ECUDA, "cuTensorMapEncodeTiled failed (%d) for S = %d", (int)r, S);
  return RIX_OK;
}

template <int MODE>
size_t fp_smem() {
  return 128 + (size_t)(MODE == kResid ? 2 : 1) * kTileBytes + (size_t)kFpWarps * sizeof(WarpScratch) +
         kCbMax * sizeof(uint32_t) + 8 + 16;
}

// resident CTAs per SM of the gridder: the job's tuning (0: the occupancy
// limit), never above it
template <int MODE, bool BATCH>
int gridder_blocks(const Ctx* ctx, int ctas_per_sm, int64_t items, size_t sm, int64_t* blocks) {
  auto kern = k_tiles_fp<MODE, BATCH>;
  RIX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  RIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFpThreads, sm));
  per_sm = std::max(per_sm, 1);
  if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
  *blocks = std::min<int64_t>(items, (int64_t)ctx->num_sms * per_sm);
  return RIX_OK;
}

template <int MODE>
int launch_fp(const Job* job, const FpArgs& a, const CUtensorMap& tm_model, const CUtensorMap& tm_out,
              cudaStream_t st) {
  const size_t sm = fp_smem<MODE>();
  int64_t blocks = 0;
  RIX_TRY((gridder_blocks<MODE, false>(job->ctx, job->fp_ctas_per_sm, a.item_count, sm, &blocks)));
  if (blocks <= 0) return RIX_OK;
  timing_mark(kTimeTiles, st, true);
  ::rix::note_launch();
  k_tiles_fp<MODE, false><<<(unsigned)blocks, kFpThreads, sm, st>>>(a, tm_model, tm_out, FpBatch{});
  timing_mark(kTimeTiles, st, false);
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

FpArgs fp_args(const Job* job, int64_t item_begin, int64_t item_count, int win_lo) {
  FpArgs a{};
  a.keys = job->keys.as<uint32_t>();
  a.items = job->items.as<uint32_t>();
  a.item_chunk = job->item_chunk.as<uint32_t>();
  a.chunks = job->chunks.as<uint32_t>();
  a.geom = job->egeom.as<float4>();
  a.ysamp = job->ysamp.as<float4>();
  a.item_begin = item_begin;
  a.item_count = item_count;
  a.bt = job->bt;
  a.bw = job->bw;
  a.win_lo = win_lo;
  a.status = job->status.as<int>();
  return a;
}

}  // namespace

int gather_y(const Job* job, int64_t ent_begin, int64_t ent_count, const void* vis, cudaStream_t st) {
  if (ent_count <= 0) return RIX_OK;
  const int blocks = (int)std::min<int64_t>(ceil_div(ent_count, 256), (int64_t)job->ctx->num_sms * 8);
  ::rix::note_launch();
  k_gather_y<<<blocks, 256, 0, st>>>(job->gsamples.as<uint32_t>(), static_cast<const float2*>(vis),
                                     job->weight.as<float>(), ent_begin, ent_count, job->ysamp.as<float4>());
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

int launch_tiles_fp(const Job* job, int mode, int64_t item_begin, int64_t item_count, int64_t ent_begin,
                    int64_t ent_count, int win_lo, int S, const void* model_planes, void* out_planes, const void* vis,
                    cudaStream_t st) {
  if (item_count <= 0 || ent_count <= 0) return RIX_OK;
  if (job->tile != kT || job->nw < kW || job->fp64 || (mode != kGrid && mode != kResid) || (S & 1))
    return set_error(RIX_EINVAL, "k_tiles_fp: unsupported job (tile %d, planes %d)", job->tile, job->nw);
  const FpArgs a = fp_args(job, item_begin, item_count, win_lo);
  CUtensorMap tm_out, tm_model;
  RIX_TRY(plane_map(&tm_out, out_planes, S, job->nw));
  // the weighted visibilities of the partition's entries in gridder order
  RIX_TRY(gather_y(job, ent_begin, ent_count, vis, st));
  if (mode == kResid) {
    RIX_TRY(plane_map(&tm_model, model_planes, S, job->nw));
    return launch_fp<kResid>(job, a, tm_model, tm_out, st);
  }
  return launch_fp<kGrid>(job, a, tm_out, tm_out, st);
}

int launch_psf_fp(const Job* job, int p, double scale, double half, void* planes, cudaStream_t st) {
  const Part& pt = job->part[p];
  const int64_t n = pt.ent_count;
  if (n <= 0 || pt.item_count <= 0) return RIX_OK;
  if (job->tile != kT || job->nw < kW || job->fp64)
    return set_error(RIX_EINVAL, "PSF gridding on k_tiles_fp: unsupported job (tile %d, planes %d)", job->tile,
                     job->nw);
  const int ntile = (pt.pwin_n + kT - 1) / kT;
  int bt = 1;
  while ((1 << bt) < ntile) ++bt;
  const int key_bits = 2 * bt + job->bw;
  if (key_bits > 32) return set_error(RIX_EINVAL, "PSF window too large for the tile keys");
  // scratch: two geometry-sized arrays (16 B per entry), ten of 4 B, three
  // lists of n + 1, four totals
  const size_t nn = (size_t)n;
  const size_t bytes = nn * 16 * 2 + nn * 4 * 10 + (nn + 1) * 4 * 3 + 16;
  unsigned char* buf = nullptr;
  if (malloc_async(&buf, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return set_error(RIX_ENOMEM, "PSF gridder scratch (%zu bytes)", bytes);
  }
  float4* geom0 = reinterpret_cast<float4*>(buf);   // image order
  float4* geom = geom0 + nn;                         // key order, then gridder order
  float4* ys = geom0;                                // unit visibilities, once geom0 is gathered
  uint32_t* key = reinterpret_cast<uint32_t*>(geom + nn);
  uint32_t* keyt = key + nn;
  uint32_t* val = keyt + nn;
  uint32_t* valt = val + nn;
  uint32_t* f = valt + nn;        // run flags, then chunk flags
  uint32_t* ex = f + nn;          // their scans
  uint32_t* starts = ex + nn;     // run starts
  float* w = reinterpret_cast<float*>(starts + nn);
  uint32_t* iflag = reinterpret_cast<uint32_t*>(w + nn);
  uint32_t* iex = iflag + nn;
  uint32_t* items = iex + nn;
  uint32_t* chunks = items + nn + 1;
  uint32_t* item_chunk = chunks + nn + 1;
  uint32_t* totals = item_chunk + nn + 1;   // runs, items, chunks
  int rc = RIX_OK;
  do {
    PsfArgs a{};
    a.keys = job->keys.as<uint32_t>();
    a.samples = job->gsamples.as<uint32_t>();
    a.uvw = job->uvw.as<double>();
    a.inv_lambda = job->inv_lambda.as<double>();
    a.nchan = job->desc.nchan;
    a.scale = scale;
    a.half = half;
    a.nw = job->nw;
    a.ww = job->ww;
    a.w_min = job->stats.w_min;
    a.dw = job->stats.dw;
    a.bt_img = job->bt;
    a.bt = bt;
    a.bw = job->bw;
    a.win_lo = pt.pwin_lo;
    a.win_n = pt.pwin_n;
    a.e_begin = pt.ent_begin;
    a.n = n;
    a.status = job->status.as<int>();
    const int eb = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)job->ctx->num_sms * 16);
    ::rix::note_launch();
    k_psf_geom<<<eb, 256, 0, st>>>(a, geom0, key, val);
    if (cudaGetLastError() != cudaSuccess) { rc = set_error(RIX_ECUDA, "k_psf_geom launch"); break; }
    // stable sort by (w-plane block, tile row, tile column)
    bool in_tmp = false;
    if ((rc = radix_sort_u32(key, val, keyt, valt, n, key_bits, st, &in_tmp)) != RIX_OK) break;
    const uint32_t* sk = in_tmp ? keyt : key;
    const uint32_t* sv = in_tmp ? valt : val;
    ::rix::note_launch();
    k_psf_runs<<<eb, 256, 0, st>>>(sk, n, f);
    if ((rc = scan_exclusive_u32(f, ex, n, totals, st)) != RIX_OK) break;
    ::rix::note_launch();
    k_psf_run_starts<<<eb, 256, 0, st>>>(f, ex, n, starts);
    ::rix::note_launch();
    k_psf_gather<<<eb, 256, 0, st>>>(sv, geom0, job->gsamples.as<uint32_t>(), job->weight.as<float>(),
                                     pt.ent_begin, f, ex, starts, n, geom, w, iflag);
    if ((rc = scan_exclusive_u32(iflag, iex, n, totals + 1, st)) != RIX_OK) break;
    ::rix::note_launch();
    k_psf_items<<<eb, 256, 0, st>>>(iflag, iex, n, totals + 1, items);
    if (cudaGetLastError() != cudaSuccess) { rc = set_error(RIX_ECUDA, "PSF work-item launches"); break; }
    {
      const size_t sm = (size_t)kItemMax * (sizeof(float4) + 2 * sizeof(uint32_t));
      if (cudaFuncSetAttribute(k_psf_order, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
        rc = set_error(RIX_ECUDA, "k_psf_order shared memory");
        break;
      }
      ::rix::note_launch();
      k_psf_order<<<job->ctx->num_sms * 4, 256, sm, st>>>(items, totals + 1, w, geom, ys, f,
                                                         std::min(std::max(job->chunk_limit, 1), kChunkLimitMax));
      if (cudaGetLastError() != cudaSuccess) { rc = set_error(RIX_ECUDA, "k_psf_order launch"); break; }
    }
    if ((rc = scan_exclusive_u32(f, ex, n, totals + 2, st)) != RIX_OK) break;
    ::rix::note_launch();
    k_psf_lists<<<eb, 256, 0, st>>>(f, ex, n, items, totals + 1, totals + 2, chunks, item_chunk);
    if (cudaGetLastError() != cudaSuccess) { rc = set_error(RIX_ECUDA, "k_psf_lists launch"); break; }
    FpArgs fa{};
    fa.keys = sk;
    fa.items = items;
    fa.item_chunk = item_chunk;
    fa.chunks = chunks;
    fa.geom = geom;
    fa.ysamp = ys;
    fa.item_begin = 0;
    fa.item_count = n;              // bounds the work items, counted on the device
    fa.dev_items = totals + 1;
    fa.bt = bt;
    fa.bw = job->bw;
    fa.win_lo = 0;                  // the keys count tiles from the window
    fa.status = job->status.as<int>();
    CUtensorMap tm{};
    if ((rc = plane_map(&tm, planes, pt.pwin_n, job->nw)) != RIX_OK) break;
    rc = launch_fp<kGrid>(job, fa, tm, tm, st);
  } while (0);
  cudaFreeAsync(buf, st);
  return rc;
}

// ---- several partitions in one launch ----------------------------------------
int batch_build(Batch* b) {
  const int n = b->n;
  std::vector<FpArgs> descs(n);
  std::vector<CUtensorMap> maps(2 * n);
  std::vector<int64_t> start(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const Job* job = b->jobs[i];
    const Part& pt = job->part[b->parts[i]];
    if (job->tile != kT || job->nw < kW || job->fp64)
      return set_error(RIX_EINVAL, "batched gridding needs FP32 w-stacked jobs with tile 16");
    descs[i] = fp_args(job, pt.item_begin, pt.item_count, pt.win_lo);
    RIX_TRY(plane_map(&maps[2 * i], pt.model_planes.p, pt.win_n, job->nw));
    RIX_TRY(plane_map(&maps[2 * i + 1], pt.resid_planes.p, pt.win_n, job->nw));
    start[i + 1] = start[i] + (pt.ent_count > 0 ? pt.item_count : 0);
  }
  b->total_items = start[n];
  RIX_TRY(b->descs.alloc(b->ctx, n * sizeof(FpArgs)));
  RIX_TRY(b->maps.alloc(b->ctx, 2 * n * sizeof(CUtensorMap)));
  RIX_TRY(b->item_start.alloc(b->ctx, (n + 1) * sizeof(int64_t)));
  RIX_CUDA(cudaMemcpy(b->descs.p, descs.data(), n * sizeof(FpArgs), cudaMemcpyHostToDevice));
  RIX_CUDA(cudaMemcpy(b->maps.p, maps.data(), 2 * n * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
  RIX_CUDA(cudaMemcpy(b->item_start.p, start.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  return RIX_OK;
}

int batch_gridder(const Batch* b, cudaStream_t st) {
  if (b->total_items <= 0) return RIX_OK;
  const size_t sm = fp_smem<kResid>();
  int64_t blocks = 0;
  RIX_TRY((gridder_blocks<kResid, true>(b->ctx, b->ctas_per_sm, b->total_items, sm, &blocks)));
  FpBatch bt{b->descs.as<FpArgs>(), b->maps.as<CUtensorMap>(), b->item_start.as<int64_t>(), b->n};
  CUtensorMap unused{};
  timing_mark(kTimeTiles, st, true);
  ::rix::note_launch();
  k_tiles_fp<kResid, true><<<(unsigned)blocks, kFpThreads, sm, st>>>(FpArgs{}, unused, unused, bt);
  timing_mark(kTimeTiles, st, false);
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

template <typename R>
int grid_work_order(Job* job, cudaStream_t st) {
  const int64_t n_ent = job->n_entries, n_items = job->n_items;
  RIX_TRY(job->gsamples.alloc(job->ctx, (size_t)std::max<int64_t>(n_ent, 1) * sizeof(uint32_t)));
  if (!job->fp64 && job->nw > 0)   // the FP32 w-stacked gridder's per-entry weighted visibilities
    RIX_TRY(job->ysamp.alloc(job->ctx, (size_t)std::max<int64_t>(n_ent, 1) * sizeof(float4)));
  RIX_TRY(job->chunks.alloc(job->ctx, (size_t)(n_ent + 1) * sizeof(uint32_t)));
  RIX_TRY(job->item_chunk.alloc(job->ctx, (size_t)(n_items + 1) * sizeof(uint32_t)));
  if (n_ent == 0 || n_items == 0) {
    RIX_CUDA(cudaMemsetAsync(job->chunks.p, 0, sizeof(uint32_t), st));
    RIX_CUDA(cudaMemsetAsync(job->item_chunk.p, 0, (size_t)(n_items + 1) * sizeof(uint32_t), st));
    return RIX_OK;
  }
  uint32_t *cflag = nullptr, *cidx = nullptr, *total = nullptr;
  int rc = RIX_OK;
  if (malloc_async(&cflag, n_ent * sizeof(uint32_t), st) != cudaSuccess ||
      malloc_async(&cidx, n_ent * sizeof(uint32_t), st) != cudaSuccess ||
      malloc_async(&total, sizeof(uint32_t), st) != cudaSuccess) {
    cudaGetLastError();
    rc = set_error(RIX_ENOMEM, "gridder order scratch");
  }
  if (rc == RIX_OK) {
    const size_t sm = (size_t)kItemMax * (sizeof(EntryGeom<R>) + 2 * sizeof(uint32_t));
    auto kern = k_item_order<R>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
      rc = set_error(RIX_ECUDA, "k_item_order shared memory");
    } else {
      const int blocks = (int)std::min<int64_t>(n_items, (int64_t)job->ctx->num_sms * 4);
      ::rix::note_launch();
      // the geometry is in the sorted order right after partitioning, in the
      // gridder order (with gsamples) when the chunks are rebuilt
      const uint32_t* in = job->gorder ? job->gsamples.as<uint32_t>() : job->samples.as<uint32_t>();
      kern<<<blocks, 256, sm, st>>>(job->items.as<uint32_t>(), n_items, in,
                                    job->egeom.as<EntryGeom<R>>(), job->gsamples.as<uint32_t>(), cflag,
                                    std::min(std::max(job->chunk_limit, 1), kChunkLimitMax));
      if (cudaGetLastError() != cudaSuccess) rc = set_error(RIX_ECUDA, "k_item_order launch");
    }
  }
  if (rc == RIX_OK) rc = scan_exclusive_u32(cflag, cidx, n_ent, total, st);
  if (rc == RIX_OK) {
    const int blocks = (int)std::min<int64_t>(ceil_div(std::max(n_ent, n_items), 256), (int64_t)job->ctx->num_sms * 8);
    ::rix::note_launch();
    k_chunk_lists<<<blocks, 256, 0, st>>>(cflag, cidx, n_ent, job->items.as<uint32_t>(), n_items, total,
                                          job->chunks.as<uint32_t>(), job->item_chunk.as<uint32_t>());
    if (cudaGetLastError() != cudaSuccess) rc = set_error(RIX_ECUDA, "k_chunk_lists launch");
  }
  if (cflag) cudaFreeAsync(cflag, st);
  if (cidx) cudaFreeAsync(cidx, st);
  if (total) cudaFreeAsync(total, st);
  if (rc == RIX_OK) job->gorder = true;
  return rc;
}

template int grid_work_order<float>(Job*, cudaStream_t);
template int grid_work_order<double>(Job*, cudaStream_t);

}  // namespace rix
