// Streamed vertex-star patch solve (persistent, TMA-fed).
//
// Each patch's factor values are contiguous in global memory and are consumed
// in a fixed order that depends only on the patch class: the forward solve
// reads the level-0 diagonal, the level-0 off-diagonal block (ELL slices), the
// level-1 line inverses, the rows of L21 and of Z = L_top^{-1}; the backward
// solve reads Z, L21, the lines and the ELL slices again in reverse.  That
// order is cut into chunks (a per-class schedule built on the host) and every
// chunk is fetched with one 1D bulk copy (cp.async.bulk) into a ring of
// shared-memory buffers, completion tracked by an mbarrier per buffer.  One
// thread keeps the ring full across patch boundaries, so the copies run
// ahead of the solve and the solve itself reads shared memory only.  The
// interface residual is gathered from the condensed cell-local FDM residual
// at the start of each patch, and only the interface solution is written.
//
// Waits on the mbarriers are bounded (a %globaltimer limit); a wait that runs
// out sets the status word, the CTA waits (again bounded) for its own copies
// in flight and returns.
#include "bulk.cuh"
#include "device.cuh"
#include "kernels.h"

namespace fdm {

namespace {

using namespace bulk;

template <typename T> struct V4s { T x, y, z, w; };
__device__ __forceinline__ V4s<float> ld4(const float *p) {
  float4 v = *reinterpret_cast<const float4 *>(p);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4s<double> ld4(const double *p) {
  double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
  return {a.x, a.y, b.x, b.y};
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
template <int NT>
__device__ __forceinline__ void consumer_sync() {  // named barrier over the NT consumer threads
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

}  // namespace

// Block = NT consumer threads + one producer warp.  full[b] completes when
// the bulk copy into ring slot b has landed; empty[b] when the consumers have
// finished reading it.
template <typename T, int NT, int MINB>
__global__ void __launch_bounds__(NT + 32, MINB) k_patch_stream(StreamArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_[];
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Grid &g = a.g;
  const int n3 = g.n * g.n * g.n;
  const int nbuf = a.nbuf;
  unsigned char *bufs = smem_;
  uint64_t *full = reinterpret_cast<uint64_t *>(bufs + (size_t)nbuf * a.buf_bytes);
  uint64_t *empty = full + nbuf;
  uint64_t *never = empty + nbuf;  // test hook: completed by nobody
  T *gv = reinterpret_cast<T *>(never + 1);
  T *yv = gv + a.maxG, *xv = yv + a.maxG, *d0 = xv + a.maxG, *acc0 = d0 + a.maxN0, *t1 = acc0 + a.maxN0;
  T *scr = t1 + a.maxN1;
  int *cur = reinterpret_cast<int *>(scr + a.tmpcap);
  __shared__ int sCell[8];
  __shared__ volatile int sFail;
  __shared__ long long sConsumed;

  if (tid == 0) {
    for (int b = 0; b < nbuf; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1);
    }
    mbar_init(never, 1);
    fence_mbar_init();
    sFail = 0;
    sConsumed = 0;
  }
  __syncthreads();

  if (warp == NW) {  // ---------------- producer warp
    if (lane == 0) {
      long long k = 0;
      bool ok = true;
      for (int q = blockIdx.x; q < a.npatch && ok; q += gridDim.x) {
        const PatchDev P = a.patches[a.order[q]];
        const ClassDev &C = a.cls[P.cls];
        const ChunkDev *sch = sizeof(T) == 4 ? C.sched32 : C.sched64;
        const int ns = sizeof(T) == 4 ? C.nsched32 : C.nsched64;
        const T *src = a.L + P.voff;
        for (int c = 0; c < ns; ++c, ++k) {
          const int b = (int)(k % nbuf);
          if (k >= nbuf && !mbar_wait_bounded(&empty[b], (uint32_t)(((k / nbuf) - 1) & 1), a.timeout_ns)) {
            ok = false;
            break;
          }
          if (sFail) { ok = false; break; }
          const ChunkDev ch = sch[c];
          fence_proxy_async();
          mbar_arrive_expect_tx(&full[b], (uint32_t)ch.bytes);
          bulk_g2s(bufs + (size_t)b * a.buf_bytes, src + ch.off, (uint32_t)ch.bytes, &full[b]);
        }
      }
      if (!ok) {
        sFail = 1;
        // wait (bounded) for the copies issued but not consumed, then leave
        for (long long j = sConsumed; j < k; ++j)
          mbar_wait_bounded(&full[j % nbuf], (uint32_t)((j / nbuf) & 1), a.timeout_ns);
        atomicExch(a.status, 1);
      }
    }
    return;
  }

  // ---------------- consumers
  if (a.inject_stall) {  // failure-detection test: wait on a barrier nothing completes
    if (!mbar_wait_bounded(never, 0, a.timeout_ns)) sFail = 1;
  }
  long long k = 0;
  for (int q = blockIdx.x; q < a.npatch; q += gridDim.x) {
    consumer_sync<NT>();
    if (sFail) break;
    const PatchDev P = a.patches[a.order[q]];
    const ClassDev &C = a.cls[P.cls];
    const int nG = C.nG, n0 = C.n0, n1 = C.n1, n2 = C.n2, base = n0 + n1;
    const ChunkDev *sch = sizeof(T) == 4 ? C.sched32 : C.sched64;
    const int ns = sizeof(T) == 4 ? C.nsched32 : C.nsched64;
    for (int i = tid; i < 3 * a.maxG; i += NT) gv[i] = T(0);
    if (tid < 8) {
      int s[3] = {tid & 1, (tid >> 1) & 1, tid >> 2};
      int ncl[3] = {g.nx, g.ny, g.nz}, cc[3];
      bool okc = true;
      for (int ax = 0; ax < 3; ++ax) {
        if (!C.full[ax] && s[ax]) okc = false;
        cc[ax] = star_cell_along(C.full[ax], P.v[ax], ncl[ax], s[ax]);
      }
      sCell[tid] = okc ? cc[0] + g.nx * (cc[1] + g.ny * cc[2]) : -1;
    }
    for (int i = tid; i < n1; i += NT) t1[i] = T(0);
    consumer_sync<NT>();
    // condensed interface residual: sum over the star cells holding each dof
    for (int kk = tid; kk < nG; kk += NT) {
      const int *src = C.gsrc + 8 * kk;
      T r = 0;
      for (int e = 0; e < 8; ++e) {
        int code = src[e];
        if (code < 0) break;
        r += a.E[(int64_t)sCell[code >> 16] * n3 + (code & 0xffff)];
      }
      gv[kk] = r;
    }
    consumer_sync<NT>();

    for (int c = 0; c < ns; ++c, ++k) {
      const ChunkDev ch = sch[c];
      const int b = (int)(k % nbuf);
      if (!mbar_wait_bounded(&full[b], (uint32_t)((k / nbuf) & 1), a.timeout_ns)) sFail = 1;
      consumer_sync<NT>();
      if (sFail) break;
      const T *buf = reinterpret_cast<const T *>(bufs + (size_t)b * a.buf_bytes);
      const int kind = ch.kind & 0xff;
      const bool first = (ch.kind >> 8) & 1, last = (ch.kind >> 9) & 1;
      switch (kind) {
        case CK_DINV:
          for (int j = tid; j < n0; j += NT) {
            T dj = buf[j];
            d0[j] = dj;
            yv[j] = gv[j] * dj;
            acc0[j] = yv[j];
            cur[j] = C.c0_ptr[j + 1];
          }
          break;
        case CK_ELL_F: {  // g_{>0} -= L_{>0,0} y_0 over the chunk's ELL slices
          const int e0 = ch.a0, e1 = ch.a1;
          for (int r = tid; r < C.nrow0; r += NT) {
            T acc = 0;
            for (int e = e0; e < e1; ++e) {
              int col = C.ell_col[e * C.ldr0 + r];
              if (col >= 0) acc += buf[(e - e0) * C.ldr0 + r] * yv[col];
            }
            gv[n0 + r] -= acc;
          }
          break;
        }
        case CK_LINES_F: {  // y_1 = L_11^{-1} g_1 for the chunk's lines
          const int b0 = ch.a0, b1 = ch.a1;
          const int i0 = C.line_start[b0], i1 = C.line_start[b1 - 1] + C.line_len[b1 - 1];
          const int lbase = C.line_off[b0];
          for (int i = i0 + tid; i < i1; i += NT) {
            int bl = C.line_of[i], s0 = C.line_start[bl], w = C.line_len[bl];
            const T *Li = buf + (C.line_off[bl] - lbase) + (i - s0) * w;
            T acc = 0;
            for (int cc = 0; cc <= i - s0; ++cc) acc += Li[cc] * gv[n0 + s0 + cc];
            yv[n0 + i] = acc;
          }
          break;
        }
        case CK_L21_F: {  // g_2 -= L21 y_1, one warp per row
          const int ng = C.ld21 / 4;
          for (int r = ch.a0 + warp; r < ch.a1; r += NW) {
            const T *row = buf + (int64_t)(r - ch.a0) * C.ld21;
            T acc = 0;
            for (int q4 = lane; q4 < ng; q4 += 32) {
              V4s<T> v = ld4(row + 4 * q4);
              const T *yy = yv + n0 + 4 * q4;
              acc += v.x * yy[0] + v.y * yy[1] + v.z * yy[2] + v.w * yy[3];
            }
            acc = warp_sum(acc);
            if (lane == 0) gv[base + r] -= acc;
          }
          break;
        }
        case CK_Z_F: {  // y_2 = Z g_2, one warp per row
          const int z0 = C.zoff[ch.a0];
          for (int r = ch.a0 + warp; r < ch.a1; r += NW) {
            const T *row = buf + (C.zoff[r] - z0);
            const int ng = (C.zoff[r + 1] - C.zoff[r]) / 4;
            T acc = 0;
            for (int q4 = lane; q4 < ng; q4 += 32) {
              V4s<T> v = ld4(row + 4 * q4);
              const T *gg = gv + base + 4 * q4;
              acc += v.x * gg[0] + v.y * gg[1] + v.z * gg[2] + v.w * gg[3];
            }
            acc = warp_sum(acc);
            if (lane == 0) yv[base + r] = acc;
          }
          break;
        }
        case CK_Z_B: {  // x_2 = Z^T y_2: (column group, row slice) partial sums
          const int ngz = (n2 + 3) / 4, ldz = 4 * ngz;
          const int slices = max(1, min(NT / ngz, a.tmpcap / ldz));
          const int gq = tid % ngz, sl = tid / ngz;
          if (sl < slices) {
            T *dst = scr + sl * ldz + 4 * gq;
            if (first) dst[0] = dst[1] = dst[2] = dst[3] = T(0);
            T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            const int z0 = C.zoff[ch.a0];
            for (int r = ch.a0 + sl; r < ch.a1; r += slices) {
              if (r < 4 * gq) continue;  // Z[r][c] = 0 for c > r
              V4s<T> v = ld4(buf + (C.zoff[r] - z0) + 4 * gq);
              T yr = yv[base + r];
              a0 += v.x * yr; a1 += v.y * yr; a2 += v.z * yr; a3 += v.w * yr;
            }
            dst[0] += a0; dst[1] += a1; dst[2] += a2; dst[3] += a3;
          }
          if (last) {
            consumer_sync<NT>();
            for (int cc = tid; cc < n2; cc += NT) {
              T s = 0;
              for (int q2 = 0; q2 < slices; ++q2) s += scr[q2 * ldz + cc];
              xv[base + cc] = s;
            }
          }
          break;
        }
        case CK_L21_B: {  // t_1 = L21^T x_2
          const int ng = C.ld21 / 4;
          const int slices = max(1, min(NT / ng, a.tmpcap / C.ld21));
          const int gq = tid % ng, sl = tid / ng;
          if (sl < slices) {
            T *dst = scr + sl * C.ld21 + 4 * gq;
            if (first) dst[0] = dst[1] = dst[2] = dst[3] = T(0);
            T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            for (int r = ch.a0 + sl; r < ch.a1; r += slices) {
              V4s<T> v = ld4(buf + (int64_t)(r - ch.a0) * C.ld21 + 4 * gq);
              T xr = xv[base + r];
              a0 += v.x * xr; a1 += v.y * xr; a2 += v.z * xr; a3 += v.w * xr;
            }
            dst[0] += a0; dst[1] += a1; dst[2] += a2; dst[3] += a3;
          }
          if (last) {
            consumer_sync<NT>();
            for (int cc = tid; cc < n1; cc += NT) {
              T s = 0;
              for (int q2 = 0; q2 < slices; ++q2) s += scr[q2 * C.ld21 + cc];
              t1[cc] = s;
            }
          }
          break;
        }
        case CK_LINES_B: {  // x_1 = L_11^{-T} (y_1 - t_1)
          const int b0 = ch.a0, b1 = ch.a1;
          const int i0 = C.line_start[b0], i1 = C.line_start[b1 - 1] + C.line_len[b1 - 1];
          const int lbase = C.line_off[b0];
          for (int i = i0 + tid; i < i1; i += NT) {
            int bl = C.line_of[i], s0 = C.line_start[bl], w = C.line_len[bl];
            const T *Lb = buf + (C.line_off[bl] - lbase);
            T s = 0;
            for (int cc = i - s0; cc < w; ++cc) s += Lb[cc * w + (i - s0)] * (yv[n0 + s0 + cc] - t1[s0 + cc]);
            xv[n0 + i] = s;
          }
          break;
        }
        case CK_ELL_B: {  // acc_0 -= L_{>0,0}^T x_{>0}, slices visited from the last
          const int e0 = ch.a0;
          for (int j = tid; j < n0; j += NT) {
            int cj = cur[j];
            T s = acc0[j];
            while (cj > C.c0_ptr[j]) {
              int pos = C.c0_pos[cj - 1];
              if (pos / C.ldr0 < e0) break;
              s -= buf[pos - e0 * C.ldr0] * xv[n0 + pos % C.ldr0];
              --cj;
            }
            acc0[j] = s;
            cur[j] = cj;
          }
          break;
        }
        default:
          break;
      }
      consumer_sync<NT>();  // slot b is free again
      if (tid == 0) {
        mbar_arrive(&empty[b]);
        sConsumed = k + 1;
      }
    }
    if (sFail) break;
    for (int j = tid; j < n0; j += NT) xv[j] = acc0[j] * d0[j];
    consumer_sync<NT>();
    T *X = a.X + P.xoff;
    for (int kk = tid; kk < nG; kk += NT) X[kk] = xv[kk];
  }
  if (sFail && tid == 0) atomicExch(a.status, 1);
}

template <typename T>
size_t stream_smem_bytes(const StreamArgs<T> &a) {
  return (size_t)a.nbuf * a.buf_bytes + 8 * (size_t)(2 * a.nbuf + 1) +
         sizeof(T) * (3 * (size_t)a.maxG + 2 * (size_t)a.maxN0 + (size_t)a.maxN1 + (size_t)a.tmpcap) +
         sizeof(int) * (size_t)a.maxN0 + 16;
}

template <typename T, int NT, int MINB>
int stream_launch_nt(const StreamArgs<T> &a0, cudaStream_t st) {
  StreamArgs<T> a = a0;
  const size_t sm = stream_smem_bytes(a);
  static size_t attr = 0;
  if (attr < sm) {
    if (cudaFuncSetAttribute(k_patch_stream<T, NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -1;
    attr = sm;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_patch_stream<T, NT, MINB>, NT + 32, sm) != cudaSuccess ||
      per_sm < 1)
    return -1;
  if (a.ctas_per_sm > 0 && a.ctas_per_sm < per_sm) per_sm = a.ctas_per_sm;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int grid = per_sm * nsm;
  if (grid > a.npatch) grid = a.npatch;
  if (grid < 1) return 0;
  k_patch_stream<T, NT, MINB><<<grid, NT + 32, sm, st>>>(a);
  return 0;
}

template <typename T>
int launch_patch_stream(const StreamArgs<T> &a, int threads, cudaStream_t st) {
  if (a.npatch <= 0) return 0;
  if (threads >= 512) return stream_launch_nt<T, 512, 1>(a, st);
  if (threads == 128) return stream_launch_nt<T, 128, 8>(a, st);
  if (a.ctas_per_sm >= 5) return stream_launch_nt<T, 256, 5>(a, st);
  return stream_launch_nt<T, 256, 2>(a, st);
}

template size_t stream_smem_bytes<float>(const StreamArgs<float> &);
template size_t stream_smem_bytes<double>(const StreamArgs<double> &);
template int launch_patch_stream<float>(const StreamArgs<float> &, int, cudaStream_t);
template int launch_patch_stream<double>(const StreamArgs<double> &, int, cudaStream_t);

}  // namespace fdm
