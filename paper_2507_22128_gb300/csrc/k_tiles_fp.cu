// a5 + a6 (Eq. 2), FP32 w-stacked: degrid, residual and grid of one uv
// partition with register-resident kernel footprints.
//
// The medium and large workloads are dense: tens of samples of one w-plane
// block fall on each uv cell, so many samples share the exact 8 x 8 x 8 tap
// footprint (same first tap in u, v and w).  At partition time the entries
// of every work item (one 16 x 16 tile of one w-plane block) are reordered by
// their first tap and cut into chunks: runs of at most 32 entries with one
// footprint.  The kernel then gives each chunk to one warp, which
//   * reads the footprint's 512 model cells from the staged tile once into
//     registers (lane: v row = lane & 7, planes lane >> 3 and that + 4, all 8
//     u taps: 16 complex cells),
//   * per sample forms the 24 kernel weights (lanes 0-23, one
//     exponential-of-semicircle evaluation each), degrids with 32 FMAs per
//     lane and a shuffle reduction, forms the weighted residual and spreads
//     it into 16 complex accumulators per lane, all in registers,
//   * adds its accumulators into the shared-memory grid tile once per chunk
//     (shared-memory float reductions: warps of one item may share cells).
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
constexpr int kChunkMax = 32;                 // entries per chunk
constexpr int kItemMax = 2048;                // entries per work item (the partition's item split)
constexpr int kFpThreads = 256;
constexpr int kFpWarps = kFpThreads / 32;
constexpr uint32_t kWaitPolls = 1u << 24;     // bounded mbarrier wait
static_assert(kTileBytes % 128 == 0, "tile alignment");

// ------------------------------------------------------ partition time -----
// Per work item: reorder its entries (at most 2048) by first tap, stably
// (key = tap << 11 | position), write the sample index of each entry in that
// order to gsamples and the geometry records in place, and flag the entries
// that start a chunk (the first of a run of one tap, and every 32nd after).
template <typename R>
__global__ void __launch_bounds__(256) k_item_order(const uint32_t* __restrict__ items, int64_t n_items,
                                                    const uint32_t* __restrict__ samples, EntryGeom<R>* geom,
                                                    uint32_t* __restrict__ gsamples, uint32_t* __restrict__ cflag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EntryGeom<R>* sg = reinterpret_cast<EntryGeom<R>*>(smem_raw);
  uint32_t* sk = reinterpret_cast<uint32_t*>(sg + kItemMax);
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const uint32_t e0 = items[item];
    const int cnt = (int)(items[item + 1] - e0);
    int p2 = 2;
    while (p2 < cnt) p2 <<= 1;
    for (int r = threadIdx.x; r < p2; r += blockDim.x) {
      if (r < cnt) {
        const EntryGeom<R> g = geom[e0 + r];
        sg[r] = g;
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
      gsamples[e0 + r] = samples[e0 + src];
      geom[e0 + r] = sg[src];
      // position of the first entry with this tap (lower bound of tap << 11)
      const uint32_t lo_key = key & ~2047u;
      int lo = 0, hi = r;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sk[mid] < lo_key) lo = mid + 1;
        else hi = mid;
      }
      cflag[e0 + r] = ((r - lo) % kChunkMax) == 0 ? 1u : 0u;
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
  const uint32_t* samples;     // sample index per entry, gridder order
  const float4* geom;          // EntryGeom<float> per entry, gridder order
  const float2* vis;           // per sample
  const float* weight;         // per sample, or null (= 1)
  int64_t item_begin, item_count;
  int bt, bw, win_lo;
  int* status;                 // the job's status word
};

constexpr unsigned kFull = 0xffffffffu;

template <int MODE>
__global__ void __launch_bounds__(kFpThreads, 2)
    k_tiles_fp(FpArgs a, const __grid_constant__ CUtensorMap tm_model, const __grid_constant__ CUtensorMap tm_out) {
  constexpr bool kModel = (MODE == kResid);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* grid = reinterpret_cast<float*>(base);
  const float2* model = reinterpret_cast<const float2*>(base + kTileBytes);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + (kModel ? 2 : 1) * kTileBytes);
  float* wscr = reinterpret_cast<float*>(bar + 2);   // per warp: two slots of 32 weights

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vrow = lane & 7, pa = lane >> 3;         // this lane's v row and planes pa, pa + 4
  const uint32_t bar_a = smem_u32(bar);
  const uint32_t tmask = (1u << a.bt) - 1u;
  if (kModel && threadIdx.x == 0) {
    mbar_init(bar_a, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  float* ws = wscr + warp * 64;

  for (int64_t it = blockIdx.x; it < a.item_count; it += gridDim.x) {
    const int64_t item = a.item_begin + it;
    const uint32_t e0 = a.items[item];
    const uint32_t key = a.keys[e0];
    const int tx = (int)(key & tmask), ty = (int)((key >> a.bt) & tmask);
    const int p0 = (int)((key >> (2 * a.bt)) & ((1u << a.bw) - 1u));
    const int u0 = tx * kT - a.win_lo, v0 = ty * kT - a.win_lo;   // >= 0: the window is tile-aligned
    if (kModel && threadIdx.x == 0) {
      mbar_expect_tx(bar_a, kTileBytes);
      tma_load_3d(smem_u32(model), &tm_model, 2 * v0, u0, p0, bar_a);
    }
    float4* g4 = reinterpret_cast<float4*>(grid);
    for (int i = threadIdx.x; i < kTileFloats / 4; i += kFpThreads) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (kModel) {
      bool ok = false;
      for (uint32_t k = 0; k < kWaitPolls && !ok; ++k) ok = mbar_try_wait(bar_a, phase);
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

    const uint32_t c0 = a.item_chunk[item], c1 = a.item_chunk[item + 1];
    for (uint32_t c = c0 + warp; c < c1; c += kFpWarps) {
      const uint32_t eb = a.chunks[c];
      const int nb = (int)(a.chunks[c + 1] - eb);
      float du = 0.f, dv = 0.f, dw = 0.f, vr = 0.f, vi = 0.f, wt = 0.f;
      uint32_t ouv = 0;
      if (lane < nb) {
        const float4 g = a.geom[eb + lane];
        du = g.x;
        dv = g.y;
        dw = g.z;
        ouv = __float_as_uint(g.w);
        const uint32_t s = a.samples[eb + lane];
        const float2 v = a.vis[s];
        wt = a.weight ? a.weight[s] : 1.0f;
        vr = wt * v.x;
        vi = wt * v.y;
      }
      ouv = __shfl_sync(kFull, ouv, 0);
      const int cell = (int)(ouv & 0xffu) * kRow + (int)(ouv >> 8) + vrow;   // complex cell in a plane
      float2 m0[kW], m1[kW];
      if (kModel) {
#pragma unroll
        for (int i = 0; i < kW; ++i) {
          m0[i] = model[pa * kPlaneC + cell + i * kRow];
          m1[i] = model[(pa + 4) * kPlaneC + cell + i * kRow];
        }
      }
      float a0r[kW], a0i[kW], a1r[kW], a1i[kW];
#pragma unroll
      for (int i = 0; i < kW; ++i) a0r[i] = a0i[i] = a1r[i] = a1i[i] = 0.f;

      for (int j = 0; j < nb; ++j) {
        // kernel weights of sample j: lanes 0-7 u taps, 8-15 v taps, 16-23 w taps
        const float kdu = __shfl_sync(kFull, du, j);
        const float kdv = __shfl_sync(kFull, dv, j);
        const float kdw = __shfl_sync(kFull, dw, j);
        const float d = lane < 8 ? kdu : (lane < 16 ? kdv : kdw);
        const float wgt = lane < 24 ? es_weight<float>(d, lane & 7) : 0.f;
        float* slot = ws + (j & 1) * 32;
        slot[lane] = wgt;
        __syncwarp();
        const float4 wlo = *reinterpret_cast<const float4*>(slot);
        const float4 whi = *reinterpret_cast<const float4*>(slot + 4);
        const float wu[kW] = {wlo.x, wlo.y, wlo.z, wlo.w, whi.x, whi.y, whi.z, whi.w};
        const float wv = slot[8 + vrow];
        const float fa = wv * slot[16 + pa], fb = wv * slot[20 + pa];
        float yr = __shfl_sync(kFull, vr, j);
        float yi = __shfl_sync(kFull, vi, j);
        if (kModel) {
          float sar = 0.f, sai = 0.f, sbr = 0.f, sbi = 0.f;
#pragma unroll
          for (int i = 0; i < kW; ++i) {
            sar = fmaf(wu[i], m0[i].x, sar);
            sai = fmaf(wu[i], m0[i].y, sai);
            sbr = fmaf(wu[i], m1[i].x, sbr);
            sbi = fmaf(wu[i], m1[i].y, sbi);
          }
          float pr = fa * sar + fb * sbr, pi = fa * sai + fb * sbi;
#pragma unroll
          for (int o = 16; o; o >>= 1) {
            pr += __shfl_xor_sync(kFull, pr, o);
            pi += __shfl_xor_sync(kFull, pi, o);
          }
          const float kwt = __shfl_sync(kFull, wt, j);
          yr = fmaf(-kwt, pr, yr);
          yi = fmaf(-kwt, pi, yi);
        }
        const float car = yr * fa, cai = yi * fa, cbr = yr * fb, cbi = yi * fb;
#pragma unroll
        for (int i = 0; i < kW; ++i) {
          a0r[i] = fmaf(car, wu[i], a0r[i]);
          a0i[i] = fmaf(cai, wu[i], a0i[i]);
          a1r[i] = fmaf(cbr, wu[i], a1r[i]);
          a1i[i] = fmaf(cbi, wu[i], a1i[i]);
        }
      }
      float* ga = grid + 2 * (pa * kPlaneC + cell);
      float* gb = grid + 2 * ((pa + 4) * kPlaneC + cell);
#pragma unroll
      for (int i = 0; i < kW; ++i) {
        atomicAdd(ga + 2 * i * kRow, a0r[i]);
        atomicAdd(ga + 2 * i * kRow + 1, a0i[i]);
        atomicAdd(gb + 2 * i * kRow, a1r[i]);
        atomicAdd(gb + 2 * i * kRow + 1, a1i[i]);
      }
    }
    // the grid tile's shared-memory writes become visible to the TMA unit,
    // then one thread adds the tile into the residual planes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      tma_reduce_add_3d(&tm_out, 2 * v0, u0, p0, smem_u32(grid));
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
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
  return 1024 + (size_t)(MODE == kResid ? 2 : 1) * kTileBytes + 16 + kFpWarps * 64 * sizeof(float);
}

template <int MODE>
int launch_fp(const Job* job, const FpArgs& a, const CUtensorMap& tm_model, const CUtensorMap& tm_out,
              cudaStream_t st) {
  const size_t sm = fp_smem<MODE>();
  auto kern = k_tiles_fp<MODE>;
  RIX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  RIX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFpThreads, sm));
  per_sm = std::max(per_sm, 1);
  const int64_t blocks = std::min<int64_t>(a.item_count, (int64_t)job->ctx->num_sms * per_sm);
  if (blocks <= 0) return RIX_OK;
  timing_mark(kTimeTiles, st, true);
  ::rix::note_launch();
  kern<<<(unsigned)blocks, kFpThreads, sm, st>>>(a, tm_model, tm_out);
  timing_mark(kTimeTiles, st, false);
  RIX_LAUNCH_CHECK();
  return RIX_OK;
}

}  // namespace

int launch_tiles_fp(const Job* job, int mode, int64_t item_begin, int64_t item_count, int win_lo, int S,
                    const void* model_planes, void* out_planes, const void* vis, cudaStream_t st) {
  if (item_count <= 0) return RIX_OK;
  if (job->tile != kT || job->nw < kW || job->fp64 || (mode != kGrid && mode != kResid) || (S & 1))
    return set_error(RIX_EINVAL, "k_tiles_fp: unsupported job (tile %d, planes %d)", job->tile, job->nw);
  FpArgs a{};
  a.keys = job->keys.as<uint32_t>();
  a.items = job->items.as<uint32_t>();
  a.item_chunk = job->item_chunk.as<uint32_t>();
  a.chunks = job->chunks.as<uint32_t>();
  a.samples = job->gsamples.as<uint32_t>();
  a.geom = job->egeom.as<float4>();
  a.vis = static_cast<const float2*>(vis);
  a.weight = job->weight.as<float>();
  a.item_begin = item_begin;
  a.item_count = item_count;
  a.bt = job->bt;
  a.bw = job->bw;
  a.win_lo = win_lo;
  a.status = job->status.as<int>();
  CUtensorMap tm_out, tm_model;
  RIX_TRY(plane_map(&tm_out, out_planes, S, job->nw));
  if (mode == kResid) {
    RIX_TRY(plane_map(&tm_model, model_planes, S, job->nw));
    return launch_fp<kResid>(job, a, tm_model, tm_out, st);
  }
  return launch_fp<kGrid>(job, a, tm_out, tm_out, st);
}

template <typename R>
int grid_work_order(Job* job, cudaStream_t st) {
  const int64_t n_ent = job->n_entries, n_items = job->n_items;
  RIX_TRY(job->gsamples.alloc(job->ctx, (size_t)std::max<int64_t>(n_ent, 1) * sizeof(uint32_t)));
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
    const size_t sm = (size_t)kItemMax * (sizeof(EntryGeom<R>) + sizeof(uint32_t));
    auto kern = k_item_order<R>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
      rc = set_error(RIX_ECUDA, "k_item_order shared memory");
    } else {
      const int blocks = (int)std::min<int64_t>(n_items, (int64_t)job->ctx->num_sms * 4);
      ::rix::note_launch();
      kern<<<blocks, 256, sm, st>>>(job->items.as<uint32_t>(), n_items, job->samples.as<uint32_t>(),
                                    job->egeom.as<EntryGeom<R>>(), job->gsamples.as<uint32_t>(), cflag);
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
  return rc;
}

template int grid_work_order<float>(Job*, cudaStream_t);
template int grid_work_order<double>(Job*, cudaStream_t);

}  // namespace rix
