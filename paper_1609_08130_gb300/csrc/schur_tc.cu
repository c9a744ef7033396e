// schur_tc.cu -- the Schur complement update of the FP32 factor on the
// tensor cores (tcgen05).
//
// After the redundant DOFs R of a box are eliminated (Sec. 2.1, Eq. 3.4),
// its skeleton-and-near block receives X_JJ -= E X_RJ with E = X_JR X_RR^{-1}
// (|J| x r) and X_RJ (r x |J|).  The rows and columns of X_JJ live in the
// pair blocks of the level (one dense block per pair of cells at Chebyshev
// distance <= 2), so the product is scattered into them.
//
// One CTA of 256 threads (two warpgroups) per (box, 128 rows of J): the E
// rows are staged in shared memory, then for every 64 columns of J the X_RJ
// columns are staged, the tile E X_RJ is accumulated in tensor memory
// (M = 128, N = 64, K = 8 per instruction) and every warp reads 32 rows x 32
// columns of it back (warp w: rows 32 (w mod 4) .., columns 32 (w / 4) ..)
// and subtracts them from the pair blocks.  54 KB of shared memory per CTA
// lets four CTAs share an SM, so many scatter loads are in flight.  FP32 accuracy is kept by splitting
// each operand into a TF32 head and an FP32 remainder: three TF32 products
// (head x head, head x remainder, remainder x head) per K step.
#include "internal.h"
#include "tc.cuh"

namespace rss {

namespace {

constexpr int TM = 128;  // rows of J per CTA (MMA M)
constexpr int TN = 64;   // columns of J per MMA tile (MMA N)
constexpr int KC = 32;   // K (= r) per staged chunk
constexpr int NTC = 256; // threads: two warpgroups over the accumulator's rows and column halves
constexpr long long WAIT_POLLS = 1ll << 20;  // polls of a bounded mbarrier wait

struct SchurTcSmem {
  static constexpr size_t A_BYTES = (size_t)TM * KC * 4;  // one of hi / lo
  static constexpr size_t B_BYTES = (size_t)TN * KC * 4;
  static constexpr size_t OPS = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr size_t TOTAL = OPS + 27 * 27 * 8 + 27 * 4 + 27 * 4 + 2 * TN * 4 + 64;
};

}  // namespace

__global__ void __launch_bounds__(NTC) k_schur_tc(LevelDev<float> lv, const FBox<float> *boxes, const int *box_list,
                                                  int row_tiles, const float *scratch, int64_t sstride, int *err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int bi = blockIdx.x / row_tiles;
  const int a0 = (blockIdx.x % row_tiles) * TM;
  const FBox<float> &fb = boxes[box_list[bi]];
  const int nj = fb.nj, r = fb.r, dim = lv.dim;
  if (r == 0 || a0 >= nj) return;
  unsigned char *opA_hi = sm, *opA_lo = sm + SchurTcSmem::A_BYTES;
  unsigned char *opB_hi = sm + 2 * SchurTcSmem::A_BYTES, *opB_lo = opB_hi + SchurTcSmem::B_BYTES;
  int64_t *s_po = reinterpret_cast<int64_t *>(sm + SchurTcSmem::OPS);
  int *s_ld = reinterpret_cast<int *>(s_po + 27 * 27);
  int *s_cell3 = s_ld + 27;
  int *s_cc = s_cell3 + 27, *s_cl = s_cc + TN;
  uint32_t *s_misc = reinterpret_cast<uint32_t *>(s_cl + TN);  // [0] TMEM base; [2..3] mbarrier (8-aligned)
  uint64_t *s_mbar = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(s_misc + 2) + 7) & ~(uintptr_t)7);

  const int tid = threadIdx.x, warp = tid >> 5;
  const float *Xrj = scratch + (int64_t)bi * sstride + (int64_t)nj * r;
  const int nc3 = dim == 3 ? 27 : 9;

  // scatter tables: pair-block offset for every (row cell, column cell) of
  // the box's 3^d neighbourhood, and the leading dimension of each row cell
  if (tid < nc3) {
    int dx, dy, dz;
    decode3(tid, dim, dx, dy, dz);
    const int cl = lv.cell_nbr[(int64_t)fb.cell * lv.NB + code5(dx, dy, dz, dim)];
    s_cell3[tid] = cl;
    s_ld[tid] = cl >= 0 ? lv.cell_b[cl] : 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_misc), TN);
  if (tid == 0) tc::mbar_init(tc::smem_u32(s_mbar), 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_misc[0];
  for (int e = tid; e < nc3 * nc3; e += NTC) {
    const int ra = e / nc3, rc = e % nc3;
    const int ca = s_cell3[ra];
    int adx, ady, adz, cdx, cdy, cdz;
    decode3(ra, dim, adx, ady, adz);
    decode3(rc, dim, cdx, cdy, cdz);
    s_po[e] = ca >= 0 ? lv.pair_off[(int64_t)ca * lv.NB + code5(cdx - adx, cdy - ady, cdz - adz, dim)] : -1;
  }
  // this thread's accumulator row (its warp's lane quarter) and column half
  const int trow = (warp & 3) * 32 + (tid & 31), chalf = warp >> 2;
  const int a = a0 + trow;
  const bool row_ok = a < nj;
  const int codea = row_ok ? fb.Jnb[a] : 0, rloc = row_ok ? fb.Jloc[a] : 0;

  const uint32_t idesc = tc::idesc_tf32(TM, TN);
  const uint32_t mbar = tc::smem_u32(s_mbar);
  const int nkc = (r + KC - 1) / KC;
  uint32_t phase = 0;
  bool ok = true;
  for (int c0 = 0; c0 < nj && ok; c0 += TN) {
    if (tid < TN) {
      const int cc = c0 + tid;
      s_cc[tid] = cc < nj ? fb.Jnb[cc] : 0;
      s_cl[tid] = cc < nj ? fb.Jloc[cc] : 0;
    }
    for (int kc = 0; kc < nkc && ok; kc++) {
      const int kw = min(KC, r - kc * KC);       // K of this chunk
      const int kp = (kw + 7) & ~7;              // padded to the MMA's K = 8
      // E rows a0.. (column-major, ld nj): staged when the chunk changes
      if (c0 == 0 || nkc > 1) {
        const int ra = a0 + (tid & (TM - 1));  // rows over the first 128 threads, again for the next
        const bool ra_ok = ra < nj;
        for (int q = tid / TM; q < kp / 4; q += NTC / TM) {
          float hv[4], lv4[4];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const int k = 4 * q + u;
            const float x = (ra_ok && k < kw) ? fb.E[ra + (int64_t)(kc * KC + k) * nj] : 0.f;
            tc::split_tf32(x, hv[u], lv4[u]);
          }
          const uint32_t o = tc::kmajor_off(tid & (TM - 1), 4 * q, TM);
          *reinterpret_cast<float4 *>(opA_hi + o) = make_float4(hv[0], hv[1], hv[2], hv[3]);
          *reinterpret_cast<float4 *>(opA_lo + o) = make_float4(lv4[0], lv4[1], lv4[2], lv4[3]);
        }
      }
      // X_RJ columns c0.. (column-major, ld r): (column, 4 consecutive k)
      // units, column fastest so the shared-memory stores do not conflict
      const int units = TN * (kp / 4);
      for (int u0 = tid; u0 < units; u0 += NTC) {
        const int n = u0 % TN, q = u0 / TN;
        const int cc = c0 + n;
        float hv[4], lv4[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int k = 4 * q + u;
          const float x = (cc < nj && k < kw) ? Xrj[(kc * KC + k) + (int64_t)cc * r] : 0.f;
          tc::split_tf32(x, hv[u], lv4[u]);
        }
        const uint32_t o = tc::kmajor_off(n, 4 * q, TN);
        *reinterpret_cast<float4 *>(opB_hi + o) = make_float4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<float4 *>(opB_lo + o) = make_float4(lv4[0], lv4[1], lv4[2], lv4[3]);
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t ah = tc::smem_u32(opA_hi), al = tc::smem_u32(opA_lo);
        const uint32_t bh = tc::smem_u32(opB_hi), bl = tc::smem_u32(opB_lo);
        for (int s = 0; s < kp / 8; s++) {
          const uint32_t oa = (uint32_t)s * TM * 32, ob = (uint32_t)s * TN * 32;
          const uint32_t acc0 = (kc > 0 || s > 0) ? 1u : 0u;
          tc::mma_tf32(tmem, tc::smem_desc(ah + oa, 128, 256), tc::smem_desc(bh + ob, 128, 256), idesc, acc0);
          tc::mma_tf32(tmem, tc::smem_desc(ah + oa, 128, 256), tc::smem_desc(bl + ob, 128, 256), idesc, 1u);
          tc::mma_tf32(tmem, tc::smem_desc(al + oa, 128, 256), tc::smem_desc(bh + ob, 128, 256), idesc, 1u);
        }
        tc::mma_commit(mbar);
      }
      // the MMAs have read the operands (and written the accumulator) once
      // the mbarrier's phase completes; a wait that gives up ends the CTA's
      // work (the same decision in every thread)
      const int late = __syncthreads_or(!tc::mbar_wait(mbar, phase, WAIT_POLLS));
      if (late) {
        if (tid == 0) set_err(err, DERR_INTERNAL);
        ok = false;
        break;
      }
      phase ^= 1u;
      tc::fence_after_sync();
    }
    if (!ok) break;
    // epilogue: this thread's row of the 128 x 64 tile, subtracted from the
    // pair blocks (column-major, ld = the row cell's level-start size); every
    // lane takes part in the warp's tensor-memory loads
    const int64_t *po_row = s_po + codea * nc3;
    const int ld = s_ld[codea];
    float *pool = lv.pool + rloc;
#pragma unroll 1
    for (int j0 = chalf * (TN / 2); j0 < (chalf + 1) * (TN / 2); j0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)j0, v);
      if (row_ok) {
#pragma unroll
        for (int j = 0; j < 16; j++) {
          if (c0 + j0 + j >= nj) break;
          float *dst = pool + po_row[s_cc[j0 + j]] + (int64_t)s_cl[j0 + j] * ld;
          if (lv.shared) atomicAdd(dst, -v[j]);  // pair blocks other boxes of the phase update too
          else *dst -= v[j];
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // accumulator read and column tables used before the next tile
    tc::fence_after_sync();
  }
  if (!ok) {
    // the MMAs of the last commit may still be running: give them one more
    // bounded wait before the tensor memory they write is freed
    tc::mbar_wait(mbar, phase, WAIT_POLLS);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, TN);
  }
}

size_t schur_tc_smem() { return SchurTcSmem::TOTAL; }

void launch_schur_tc(const LevelDev<float> &lv, const FBox<float> *boxes, const int *box_list, int nbox, int njmax,
                     const float *scratch, int64_t scratch_stride, cudaStream_t st, int *err) {
  if (nbox == 0) return;
  const int rt = (njmax + TM - 1) / TM;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
    cudaFuncSetAttribute(k_schur_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SchurTcSmem::TOTAL);
  const int64_t grid = (int64_t)nbox * rt;
  k_schur_tc<<<(unsigned)grid, NTC, SchurTcSmem::TOTAL, st>>>(lv, boxes, box_list, rt, scratch, scratch_stride, err);
  count_launch();
}

}  // namespace rss
