// les_cg_regs.cu -- the on-chip conjugate-gradient Poisson solve (Sec. 2.4:
// L_c psi = b, compact 7-point Laplacian, periodic in x and y, mirror or
// periodic in z; mean of b removed, psi returned with zero mean) for FP32
// grids 128 nodes wide, with p, r and q = L_c p held in registers.
//
// Each block of one persistent cooperative launch owns a brick spanning the
// whole x extent by `by` rows by `bz` planes for the whole solve.  Warp w
// owns brick row w mod by and one run of the brick's planes (the planes are
// split into zs runs of nearly equal length, run w / by); lane l owns the
// four consecutive nodes 4l .. 4l + 3 of each of its planes.  A thread thus
// keeps at most ZP planes x 4 nodes of p, r and q in registers, and the
// 7-point stencil finds its x neighbours in the thread's own registers and
// in the adjacent lanes (one shuffle each way; the brick spans the periodic
// x extent, so lanes 0 and 31 are neighbours), its z neighbours in the
// thread's own planes, and only its y neighbours, and the z neighbours past
// either end of its run, in a copy of p in shared memory.  That copy (with a
// one-node ghost layer in y and z), x, the last iteration's p, r at the
// ghost nodes and a staging area for the neighbours' q faces are all the
// block keeps in shared memory: an iteration touches shared memory about
// five times per node (one load of each y neighbour, one store of p, and
// x += alpha p from the kept p) instead of the sixteen accesses of a solve
// with all vectors in shared memory.
//
// An iteration (one grid-wide sum, the recurrences of the shared-memory
// solver in les_cg_resident.cu):
//   matvec   q = L_c p; the q faces a neighbour reads are published;
//            p.q, r.q and q.q (r.r was formed with r, in the update)
//   sum      each warp reduces its four values in FP32 (a transposing
//            butterfly: six shuffles for all four); warp 0 combines the
//            warps' values as compensated FP32 pairs, writes them into
//            kSpread copies and arrives on one of kSpread counters (block b
//            on counter b mod kSpread), and its lanes 0 .. kSpread - 1 wait
//            for one counter each (the grid sum of les_gridsync.cuh, with
//            its arrivals and reads spread over as many L2 lines); then
//            warps 0 .. 3 fold one value each from the block's copy, in
//            block order, while the other warps copy the neighbours' q
//            faces into shared memory asynchronously; thread 0 forms
//            alpha and beta = |r - alpha q|^2 / r.r from the totals
//   update   r -= alpha q, p = r + beta p (registers and the shared copy of
//            p); at the ghost nodes r -= alpha q_ghost and p = r + beta p;
//            x += alpha p in warp 0, while the other warps keep p and add
//            alpha p to x during the next sum's wait, when they are idle
#include <algorithm>
#include <string>

#include "les_gridsync.cuh"
#include "les_internal.h"

namespace les {
namespace {

constexpr int kRegNx = 128;       // grid width: 32 lanes x 4 nodes
constexpr int kRegMaxWarps = 16;  // 512 threads of at most 128 registers
constexpr int kSpread = 8;        // arrival counters and copies of the partials per sum
constexpr int kLineWords = 32;    // counters 128 bytes apart
static_assert(kSpread * 4 == 32, "one lane of warp 0 per (copy, value) of the partials");

struct RegArgs {
  int ny, nz, walls;
  float cx, cy, cz;  // 1/dx^2, 1/dy^2, 1/dz^2
  int by, zs;        // brick rows; runs of planes per brick
  int py, pz;        // bricks along y and z (z extents differ by at most one)
  long long n;
  const float* b;
  float* x;
  float* rg;         // published faces of the first residual
  float* qg0;        // published faces of q, even iterations
  float* qg1;        // ... odd iterations
  double* partials;  // two slots of kSumSlot words per block (the set-up and gauge sums)
  unsigned* counters;  // kSpread arrival counters of the iterations' sums, kLineWords apart, zeroed
  F2* spread;          // [2 slots][kSpread copies][4 values][gridDim.x] partials of those sums
  unsigned missing;    // test hook: arrivals on counter 0 that never come
  FusedBar* bar;
  SolverCtl* ctl;
  double tol;
  int maxit;
  long long spin_cycles;
  unsigned expected;
};

__device__ __forceinline__ int reg_zghost(int k, int nz, int walls) {
  if (walls) return k < 0 ? -1 - k : (k >= nz ? 2 * nz - 1 - k : k);
  return k < 0 ? k + nz : (k >= nz ? k - nz : k);
}
__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void stg4(float* p, float4 v) { __stcg(reinterpret_cast<float4*>(p), v); }


template <int ZP>
__global__ void __launch_bounds__(kRegMaxWarps * 32, 1) k_cg_regs(RegArgs f) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  const int by = f.by;
  const int bj = blockIdx.x % f.py, bk = blockIdx.x / f.py;
  const int zbase = f.nz / f.pz, zrem = f.nz % f.pz;
  const int bz = zbase + (bk < zrem ? 1 : 0), bzmax = zbase + (zrem ? 1 : 0);
  const int j0 = bj * by, k0 = bk * zbase + min(bk, zrem);
  // this thread's brick row and run of planes
  const int ly = warp % by, run = warp / by;
  const int zq = bz / f.zs, zr = bz % f.zs;
  const int z0 = run * zq + min(run, zr), nzp = zq + (run < zr ? 1 : 0);
  const int SZ = (by + 2) * kRegNx;  // plane stride of the haloed copy of p
  const int nr = 2 * by + 2 * bz;    // ghost rows: z faces, then y faces
  const int x4 = 4 * lane;
  float* P = reinterpret_cast<float*>(smraw);         // (bzmax + 2) x (by + 2) rows of 128
  float* X = P + (size_t)(bzmax + 2) * SZ;            // bzmax x by rows
  float* RG = X + (size_t)bzmax * by * kRegNx;        // r at the ghost rows
  float* GQ = RG + (size_t)2 * (by + bzmax) * kRegNx;  // the neighbours' q at the ghost rows
  float* PO = GQ + (size_t)2 * (by + bzmax) * kRegNx;  // p of the last iteration, as X
  const float cx = f.cx, cy = f.cy, cz = f.cz;
  // this thread's own rows: plane j of its run lies at pown + j SZ in P,
  // xown + j xpl in X and gown + j gpl in global memory (never wrapped)
  const int pown = (z0 + 1) * SZ + (ly + 1) * kRegNx + x4;
  const int xpl = by * kRegNx, xown = (z0 * by + ly) * kRegNx + x4;
  const size_t gpl = (size_t)f.ny * kRegNx;
  const size_t gown = ((size_t)(k0 + z0) * f.ny + j0 + ly) * kRegNx + x4;
  const bool frow = ly == 0 || ly == by - 1;  // a y face: every plane is read by a neighbour

  auto prow = [&](int y, int z) { return (z + 1) * SZ + (y + 1) * kRegNx; };
  // global start of brick row (y, z), at most one node outside the brick
  auto grow = [&](int y, int z) -> size_t {
    int j = j0 + y;
    j = j < 0 ? j + f.ny : (j >= f.ny ? j - f.ny : j);
    return ((size_t)reg_zghost(k0 + z, f.nz, f.walls) * f.ny + j) * kRegNx;
  };
  auto ghost_row = [&](int row, int& y, int& z) {
    if (row < 2 * by) {
      y = row >> 1;
      z = (row & 1) ? bz : -1;
    } else {
      z = (row - 2 * by) >> 1;
      y = (row & 1) ? by : -1;
    }
  };
  auto is_face = [&](int j) { return frow || z0 + j == 0 || z0 + j == bz - 1; };
  // every ghost row of A into P (and RG when keep), all warps, outside the iterations
  auto fill_ghosts = [&](const float* A, bool keep) {
    for (int row = warp; row < nr; row += nwarp) {
      int y, z;
      ghost_row(row, y, z);
      const float4 v = ldg4(A + grow(y, z) + x4);
      if (keep) sts4(RG + row * kRegNx + x4, v);
      sts4(P + prow(y, z) + x4, v);
    }
  };

  float4 p[ZP] = {}, r[ZP], q[ZP];
  // L_c p at the four nodes of plane j of this thread's run; second
  // differences formed before scaling, as in the other CG kernels
  auto stencil = [&](int j) -> float4 {
    const float4 c = p[j];
    const float w0 = __shfl_sync(0xffffffffu, c.w, (lane + 31) & 31);
    const float e3 = __shfl_sync(0xffffffffu, c.x, (lane + 1) & 31);
    const float* pj = P + pown + j * SZ;
    const float4 s = lds4(pj - kRegNx);
    const float4 nn = lds4(pj + kRegNx);
    const float4 d = j > 0 ? p[j > 0 ? j - 1 : 0] : lds4(pj - SZ);
    const float4 u = (j + 1 < ZP && j + 1 < nzp) ? p[j + 1 < ZP ? j + 1 : ZP - 1] : lds4(pj + SZ);
    auto node = [&](float pc, float pw, float pe, float ps, float pn, float pd, float pu) {
      const float c2 = 2.f * pc;
      return (pw + pe - c2) * cx + (ps + pn - c2) * cy + (pd + pu - c2) * cz;
    };
    return make_float4(node(c.x, w0, c.y, s.x, nn.x, d.x, u.x), node(c.y, c.x, c.z, s.y, nn.y, d.y, u.y),
                       node(c.z, c.y, c.w, s.z, nn.z, d.z, u.z), node(c.w, c.z, e3, s.w, nn.w, d.w, u.w));
  };

  GridSync gs{f.bar, f.partials, f.spin_cycles, f.expected, 0u};
  // set-up results of thread 0, broadcast through shared memory
  __shared__ struct {
    float mean, ta, tb;
    int status;
  } sc;
  __shared__ float shv[4][kRegMaxWarps];
  __shared__ F2 tot[4];
  __shared__ int s_fail;
  double rr = 0.0, bb = 0.0, rel = 0.0;  // meaningful in thread 0
  int status = 0;  // 0 running, 1 converged, 2 maxit, 3 breakdown, 4 zero rhs, 5 timeout
  // this thread's share of r.r for the next sum, formed where r is (the
  // initial residual, then each update), in the order the sums expect
  float rr_own = 0.f;

  // mean of b (b held in r)
  {
    Dot<float> a1[1];
#pragma unroll
    for (int j = 0; j < ZP; ++j)
      if (j < nzp) {
        r[j] = ldg4(f.b + gown + j * gpl);
        a1[0].add(r[j].x);
        a1[0].add(r[j].y);
        a1[0].add(r[j].z);
        a1[0].add(r[j].w);
      }
    double t[1];
    const bool ok = grid_dot_t0<1>(a1, gs, t);
    if (tid == 0) {
      sc.status = ok ? 0 : 5;
      sc.mean = (float)(t[0] / (double)f.n);
    }
    __syncthreads();
    status = sc.status;
  }
  const float mean = sc.mean;

  // x0 with its ghosts in p and the copy; r = (b - mean) - L_c x0, published;
  // r.r and |b - mean|^2
  if (!status) {
#pragma unroll
    for (int j = 0; j < ZP; ++j)
      if (j < nzp) {
        p[j] = ldg4(f.x + gown + j * gpl);
        sts4(X + xown + j * xpl, p[j]);
        sts4(P + pown + j * SZ, p[j]);
      }
    fill_ghosts(f.x, false);
    __syncthreads();
    Dot<float> a2[2];
#pragma unroll
    for (int j = 0; j < ZP; ++j)
      if (j < nzp) {
        const float4 l = stencil(j);
        const float4 bm = make_float4(r[j].x - mean, r[j].y - mean, r[j].z - mean, r[j].w - mean);
        r[j] = make_float4(bm.x - l.x, bm.y - l.y, bm.z - l.z, bm.w - l.w);
        if (is_face(j)) stg4(f.rg + gown + j * gpl, r[j]);
        a2[0].add(r[j].x * r[j].x);
        a2[0].add(r[j].y * r[j].y);
        a2[0].add(r[j].z * r[j].z);
        a2[0].add(r[j].w * r[j].w);
        a2[1].add(bm.x * bm.x);
        a2[1].add(bm.y * bm.y);
        a2[1].add(bm.z * bm.z);
        a2[1].add(bm.w * bm.w);
      }
    rr_own = a2[0].s;
    double s2[2];
    const bool ok = grid_dot_t0<2>(a2, gs, s2);
    if (tid == 0) {
      sc.status = ok ? 0 : 5;
      rr = s2[0];
      bb = s2[1];
    }
    __syncthreads();
    status = sc.status;
  }
  if (tid == 0) {
    if (!status) {
      if (bb == 0.0) status = 4;
      else {
        rel = sqrt(rr / bb);
        if (rel <= f.tol) status = 1;
        else if (f.maxit <= 0) status = 2;
      }
    }
    sc.status = status;
  }
  __syncthreads();
  status = sc.status;

  // the iterations: alpha = r.r / p.q, |r_{i+1}|^2 = r.r - 2 alpha r.q +
  // alpha^2 q.q, beta = |r_{i+1}|^2 / r.r from one sum of four values;
  // convergence judged on each sum's r.r against tol^2 |b - mean|^2
  __shared__ double s_bb, s_rel;  // |b - mean|^2 and the relative residual of x0
  if (tid == 0) {
    s_bb = bb;
    s_rel = rel;
  }
  __syncthreads();
  F2 rr_stop, rr_last;  // rr_last meaningful in thread 0
  acc_from(f.tol * f.tol * s_bb, rr_stop);
  acc_from(rr, rr_last);
  int iter = 0;
  float ta = 0.f, tb = 0.f;
  unsigned it_sum = 0;  // sums of the iterations completed
  if (!status) {
    // p_0 = r_0, with r_0 at the ghost nodes from the published faces
    __syncthreads();  // the initial residual's stencil reads of the copy are done
#pragma unroll
    for (int j = 0; j < ZP; ++j)
      if (j < nzp) {
        p[j] = r[j];
        sts4(P + pown + j * SZ, p[j]);
      }
    fill_ghosts(f.rg, true);
    __syncthreads();
    for (;;) {
      float* qw = (iter & 1) ? f.qg1 : f.qg0;  // this iteration's q faces
      Dot<float> d[4];                         // p.q, r.r, r.q, q.q
#pragma unroll
      for (int j = 0; j < ZP; ++j)
        if (j < nzp) {
          q[j] = stencil(j);
          if (is_face(j)) stg4(qw + gown + j * gpl, q[j]);
          d[0].add(p[j].x * q[j].x);
          d[0].add(p[j].y * q[j].y);
          d[0].add(p[j].z * q[j].z);
          d[0].add(p[j].w * q[j].w);
          d[2].add(r[j].x * q[j].x);
          d[2].add(r[j].y * q[j].y);
          d[2].add(r[j].z * q[j].z);
          d[2].add(r[j].w * q[j].w);
          d[3].add(q[j].x * q[j].x);
          d[3].add(q[j].y * q[j].y);
          d[3].add(q[j].z * q[j].z);
          d[3].add(q[j].w * q[j].w);
        }
      d[1].s = rr_own;
      // the grid sum.  Each warp's four values in FP32 by a transposing
      // butterfly: after it lanes 8k .. 8k + 7 hold the warp's value k.
      {
        const bool up = lane & 16, odd = lane & 8;
        float a0 = up ? d[2].s : d[0].s, a1 = up ? d[3].s : d[1].s;        // kept
        const float s0 = up ? d[0].s : d[2].s, s1 = up ? d[1].s : d[3].s;  // given to lane ^ 16
        a0 += __shfl_xor_sync(0xffffffffu, s0, 16);
        a1 += __shfl_xor_sync(0xffffffffu, s1, 16);
        float v = odd ? a1 : a0;
        v += __shfl_xor_sync(0xffffffffu, odd ? a0 : a1, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if ((lane & 7) == 0) shv[lane >> 3][warp] = v;
      }
      // also orders every thread's q-face stores before warp 0's release
      __syncthreads();
      const unsigned G = gridDim.x;
      // this sum's partials: kSpread copies, so that the blocks' reads of
      // them spread over as many L2 lines; this block reads copy b mod kSpread
      F2* slot = f.spread + (size_t)(it_sum & 1u) * kSpread * 4 * G;
      if (warp == 0) {
        // lanes 8k .. 8k + 7: value k of the block as a compensated pair
        const int k = lane >> 3;
        F2 a = F2{0.f, 0.f};
        for (int w = lane & 7; w < nwarp; w += 8) a = f2_add(a, F2{shv[k][w], 0.f});
#pragma unroll
        for (int o = 4; o > 0; o >>= 1)
          a = f2_add(a, F2{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)});
        // lane l writes value l mod 4 into copy l / 4
        const int src = 8 * (lane & 3);
        const F2 mine = F2{__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
        acc_store(slot + ((size_t)(lane >> 2) * 4 + (lane & 3)) * G + blockIdx.x, mine);
        // orders the lanes' stores before lane 0's release
        __syncwarp();
        if (lane == 0) red_release_add(f.counters + (blockIdx.x % kSpread) * kLineWords, 1u);
        // posted: the other warps may start on shared memory
        asm volatile("bar.arrive 2, %0;" ::"r"(nthr) : "memory");
        // lanes 0 .. kSpread - 1 wait for the arrivals on one counter each
        // (counter i takes blocks i, i + kSpread, ...; counter 0 also the
        // test hook's missing ones)
        bool done = lane >= kSpread;
        const unsigned mine_n = lane < (int)G ? (G - lane + kSpread - 1) / kSpread : 0u;
        const unsigned target = done ? 0u : (it_sum + 1u) * (mine_n + (lane == 0 ? f.missing : 0u));
        const long long t0 = clock64();
        int fail = 0;
        for (unsigned spins = 1;; ++spins) {
          if (!done) done = (int)(ld_acquire(f.counters + lane * kLineWords) - target) >= 0;
          if (__all_sync(0xffffffffu, done)) break;
          const bool quit = (spins & 63u) == 0u && (ld_volatile(&gs.bar->fail.v) != 0u || clock64() - t0 > gs.spin);
          if (__any_sync(0xffffffffu, quit)) {
            if (lane == 0) atomicExch(&gs.bar->fail.v, 1u);
            fail = 1;
            break;
          }
        }
        // orders the lanes' acquires before the reads of every lane
        __syncwarp();
        if (lane == 0) s_fail = fail;
        // every block has arrived (or the wait gave up): the other warps may
        // read the partials and the q faces published before the arrivals
        asm volatile("bar.arrive 1, %0;" ::"r"(nthr) : "memory");
      } else {
        // while warp 0 waits: the last iteration's x += alpha p of this
        // warp's rows (deferred from its update), once warp 0 has posted
        asm volatile("bar.sync 2, %0;" ::"r"(nthr) : "memory");
        if (iter > 0) {
#pragma unroll
          for (int j = 0; j < ZP; ++j)
            if (j < nzp) {
              float4 xv = lds4(X + xown + j * xpl);
              const float4 pv = lds4(PO + xown + j * xpl);
              xv.x += ta * pv.x;
              xv.y += ta * pv.y;
              xv.z += ta * pv.z;
              xv.w += ta * pv.w;
              sts4(X + xown + j * xpl, xv);
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
      }
      const F2* mycopy = slot + (size_t)(blockIdx.x % kSpread) * 4 * G;
      // warps 0 .. 3 fold one value each (in block order, so every block
      // obtains the same totals) while the others copy the ghost rows of q
      // into GQ (every warp, after its folds, in a block of four warps or
      // fewer)
      const int l0 = nwarp > 4 ? 4 : 0;
      if (warp >= l0) {
        for (int row = warp - l0; row < nr; row += nwarp - l0) {
          int y, z;
          ghost_row(row, y, z);
          cp_async_bytes<16>(GQ + row * kRegNx + x4, qw + grow(y, z) + x4);
        }
        cp_commit();
      }
      if (warp < 4) {
        for (int k = warp; k < 4; k += nwarp) {
          F2 t = F2{0.f, 0.f};
          for (unsigned b0 = lane; b0 < G; b0 += 32 * 5) {
            F2 w[5];
#pragma unroll
            for (int u = 0; u < 5; ++u)
              w[u] = b0 + 32 * u < G ? acc_load(mycopy + (size_t)k * G + b0 + 32 * u) : F2{0.f, 0.f};
#pragma unroll
            for (int u = 0; u < 5; ++u) t = f2_add(t, w[u]);
          }
          t = warp_sum_f2(t);
          if (lane == 0) tot[k] = t;
        }
        // the folds are complete: thread 0 forms the status, alpha and beta
        asm volatile("bar.sync 3, %0;" ::"r"(32 * min(nwarp, 4)) : "memory");
        if (tid == 0) {
          int st = 0;
          if (s_fail) {
            st = 5;
          } else {
            const F2 t1 = tot[1];
            rr_last = t1;
            if (acc_le(t1, rr_stop)) st = 1;
            else if (iter >= f.maxit) st = 2;
            else {
              const float pq = tot[0].hi, r2 = t1.hi, rq = tot[2].hi, q2 = tot[3].hi;
              if (!(pq != 0.f) || !isfinite(pq) || !isfinite(r2)) {
                st = 3;
              } else {
                const float alpha = r2 / pq;
                const float rn = fmaf(alpha * alpha, q2, fmaf(-2.f * alpha, rq, r2));  // |r - alpha q|^2
                sc.ta = alpha;
                sc.tb = rn / r2;
              }
            }
          }
          sc.status = st;
        }
      }
      if (!l0) {
        for (int row = warp; row < nr; row += nwarp) {
          int y, z;
          ghost_row(row, y, z);
          cp_async_bytes<16>(GQ + row * kRegNx + x4, qw + grow(y, z) + x4);
        }
        cp_commit();
      }
      cp_wait<0>();
      it_sum += 1u;
      __syncthreads();
      status = sc.status;
      if (status) break;
      ta = sc.ta;
      tb = sc.tb;
      float rr_new = 0.f;
#pragma unroll
      for (int j = 0; j < ZP; ++j)
        if (j < nzp) {
          if (warp == 0) {
            float4 xv = lds4(X + xown + j * xpl);
            xv.x += ta * p[j].x;
            xv.y += ta * p[j].y;
            xv.z += ta * p[j].z;
            xv.w += ta * p[j].w;
            sts4(X + xown + j * xpl, xv);
          } else {
            sts4(PO + xown + j * xpl, p[j]);
          }
          r[j].x -= ta * q[j].x;
          r[j].y -= ta * q[j].y;
          r[j].z -= ta * q[j].z;
          r[j].w -= ta * q[j].w;
          rr_new += r[j].x * r[j].x;
          rr_new += r[j].y * r[j].y;
          rr_new += r[j].z * r[j].z;
          rr_new += r[j].w * r[j].w;
          p[j].x = r[j].x + tb * p[j].x;
          p[j].y = r[j].y + tb * p[j].y;
          p[j].z = r[j].z + tb * p[j].z;
          p[j].w = r[j].w + tb * p[j].w;
          sts4(P + pown + j * SZ, p[j]);
        }
      for (int row = warp; row < nr; row += nwarp) {
        int y, z;
        ghost_row(row, y, z);
        const float4 gq = lds4(GQ + row * kRegNx + x4);
        float4 rv = lds4(RG + row * kRegNx + x4);
        rv.x -= ta * gq.x;
        rv.y -= ta * gq.y;
        rv.z -= ta * gq.z;
        rv.w -= ta * gq.w;
        sts4(RG + row * kRegNx + x4, rv);
        float* pg = P + prow(y, z) + x4;
        float4 pv = lds4(pg);
        pv.x = rv.x + tb * pv.x;
        pv.y = rv.y + tb * pv.y;
        pv.z = rv.z + tb * pv.z;
        pv.w = rv.w + tb * pv.w;
        sts4(pg, pv);
      }
      rr_own = rr_new;
      iter += 1;
      __syncthreads();
    }
  }
  if (tid == 0) rel = (iter > 0 && s_bb > 0.0) ? sqrt(acc_value(rr_last) / s_bb) : s_rel;

  // zero-mean gauge (or zero for a zero right side), written back to x
  if (status != 5) {
    Dot<float> ax[1];
#pragma unroll
    for (int j = 0; j < ZP; ++j)
      if (j < nzp) {
        const float4 xv = lds4(X + xown + j * xpl);
        ax[0].add(xv.x);
        ax[0].add(xv.y);
        ax[0].add(xv.z);
        ax[0].add(xv.w);
      }
    double t[1];
    const bool ok = grid_dot_t0<1>(ax, gs, t);
    if (tid == 0) {
      if (!ok) status = 5;
      sc.mean = (float)(t[0] / (double)f.n);
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
    if (status != 5) {
      const float mx = sc.mean;
#pragma unroll
      for (int j = 0; j < ZP; ++j)
        if (j < nzp) {
          const float4 xv = lds4(X + xown + j * xpl);
          stg4(f.x + gown + j * gpl, status == 4 ? make_float4(0.f, 0.f, 0.f, 0.f)
                                                   : make_float4(xv.x - mx, xv.y - mx, xv.z - mx, xv.w - mx));
        }
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    f.ctl->iter = iter;
    f.ctl->rel = rel;
    f.ctl->done = status;
  }
}

struct RegPlan {
  int by = 0, pz = 0, zs = 0, zp = 0, bz = 0;  // bz: the largest brick extent in z
  size_t smem = 0;
  long long G = 0;
};

// p with its ghost layer, x, r and the neighbours' q at the ghost rows, and
// the last iteration's p
size_t regs_smem(int by, int bz) {
  return ((size_t)(bz + 2) * (by + 2) + 2 * (size_t)bz * by + 4 * (size_t)(by + bz)) * kRegNx * sizeof(float);
}

// Bricks of the whole x extent by `by` rows (by | ny, by <= 16) by pz runs of
// z (extents rounded up or down), at most one brick per SM, split among
// by x zs warps (at most 16) with at most 6 planes per thread; among those
// the one with the fewest planes per thread, then the fewest blocks, then
// the fewest ghost rows per warp.
bool make_regs_plan(int ny, int nz, int nsm, size_t smem_max, int max_blocks, RegPlan& best) {
  const int gmax = std::min(nsm, max_blocks);
  bool found = false;
  long long bk0 = 0, bk1 = 0, bk2 = 0;
  for (int by = 1; by <= std::min(ny, kRegMaxWarps); ++by) {
    if (ny % by) continue;
    for (int pz = 1; pz <= nz; ++pz) {
      const int bz = (nz + pz - 1) / pz, zbase = nz / pz;
      if (pz > 1 && (nz + pz - 2) / (pz - 1) == bz) continue;  // as large, with more bricks
      const long long G = (long long)(ny / by) * pz;
      if (G > gmax) break;
      for (int zs = 1; by * zs <= kRegMaxWarps && zs <= zbase; ++zs) {
        const int zp = (bz + zs - 1) / zs, nw = by * zs, nr = 2 * by + 2 * bz;
        if (zp > 6) continue;
        const size_t smem = regs_smem(by, bz);
        if (smem > smem_max) continue;
        const long long k0 = zp, k1 = G, k2 = (nr + nw - 1) / nw;
        if (!found || k0 < bk0 || (k0 == bk0 && (k1 < bk1 || (k1 == bk1 && k2 < bk2)))) {
          found = true;
          bk0 = k0;
          bk1 = k1;
          bk2 = k2;
          best.by = by;
          best.pz = pz;
          best.zs = zs;
          best.zp = zp;
          best.bz = bz;
          best.smem = smem;
          best.G = G;
        }
      }
    }
  }
  return found;
}

const void* regs_kernel(int zp) {
  if (zp <= 2) return (const void*)k_cg_regs<2>;
  if (zp <= 4) return (const void*)k_cg_regs<4>;
  return (const void*)k_cg_regs<6>;
}

}  // namespace

int poisson_solve_regs(const SolverArgs<float>& a, const FusedCfg& fc, const float* b, float* x, double tol,
                       int maxit, int* iters, double* rel, std::string* err, bool* used) {
  *used = false;
  // a guarded first guess (judged against x0 = 0) is left to the
  // shared-memory kernel: the learned guess that asks for it needs a cubic
  // grid, and no 128^3 grid fits on chip
  if (!(a.op == LES_OP_COMPACT && a.solver == LES_SOLVER_CG && a.g.nx == kRegNx && a.g.nz >= 2 && !a.guard &&
        a.bar && a.r && a.p0 && a.p1))
    return LES_OK;
  int dev = 0, nsm = 0, smem_optin = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) {
    if (err) *err = std::string("register CG: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  RegPlan pl;
  // leave room for the reductions' static shared memory (about 2 KB)
  if (!make_regs_plan(a.g.ny, a.g.nz, nsm, (size_t)std::max(0, smem_optin - 3072), fc.max_blocks, pl)) return LES_OK;
  const void* kern = regs_kernel(pl.zp);
  const int nthr = 32 * pl.by * pl.zs;
  int per_sm = 0;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthr, pl.smem)) != cudaSuccess) {
    if (err) *err = std::string("register CG occupancy: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  if (per_sm < 1 || pl.G > (long long)per_sm * nsm) return LES_OK;  // not co-resident
  RegArgs f;
  f.ny = a.g.ny;
  f.nz = a.g.nz;
  f.walls = a.g.walls;
  f.cx = a.g.idx * a.g.idx;
  f.cy = a.g.idy * a.g.idy;
  f.cz = a.g.idz * a.g.idz;
  f.by = pl.by;
  f.zs = pl.zs;
  f.py = a.g.ny / pl.by;
  f.pz = pl.pz;
  f.n = (long long)kRegNx * f.ny * f.nz;
  f.b = b;
  f.x = x;
  f.rg = a.r;
  f.qg0 = a.p0;
  f.qg1 = a.p1;
  f.partials = a.partials;
  // past the set-up sums' two slots: the counters, then the copies of the
  // iterations' partials (2 x kSpread x 4 words per block)
  f.counters = reinterpret_cast<unsigned*>(a.partials + 2 * (size_t)kSumSlot * pl.G);
  f.spread = reinterpret_cast<F2*>(a.partials + 2 * (size_t)kSumSlot * pl.G + kSpread * kLineWords / 2);
  f.missing = (unsigned)std::max(0, fc.missing);
  f.bar = a.bar;
  f.ctl = a.ctl;
  f.tol = tol;
  f.maxit = maxit;
  f.spin_cycles = fc.spin_cycles;
  // the test hook's missing arrivals apply to the iterations' sums (whose
  // wait is this kernel's own); the set-up sums wait for the launched blocks
  f.expected = (unsigned)pl.G;
  *used = true;
  if ((e = cudaMemsetAsync(a.bar, 0, sizeof(FusedBar), a.st)) != cudaSuccess ||
      (e = cudaMemsetAsync(f.counters, 0, kSpread * kLineWords * sizeof(unsigned), a.st)) != cudaSuccess) {
    if (err) *err = std::string("register CG barrier reset: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  void* args[] = {&f};
  {
    ProfScope ps(a.prof, KI_CG_REGS, a.st);
    e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)pl.G), dim3(nthr), args, pl.smem, a.st);
  }
  if (e != cudaSuccess) {
    if (err) *err = std::string("register CG launch: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  if ((e = cudaMemcpyAsync(a.ctl_host, a.ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, a.st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(a.st)) != cudaSuccess) {
    if (err) *err = std::string("register CG: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  const SolverCtl& c = *a.ctl_host;
  if (iters) *iters = c.iter;
  if (rel) *rel = c.rel;
  // algorithmic traffic of the solve, as for every CG kernel (its vectors
  // stay on chip)
  if (a.prof) a.prof->bytes[KI_CG_REGS] += (kCgSetupFields + kCgIterFields * c.iter) * (double)f.n * sizeof(float);
  switch (c.done) {
    case 1:
    case 4: return LES_OK;
    case 2: return LES_ERR_NOT_CONVERGED;
    case 3:
      if (err) *err = "poisson: breakdown (zero or non-finite p.Ap / residual)";
      return LES_ERR_NONFINITE;
    case 5:
      if (err) *err = "poisson: a grid barrier wait timed out";
      return LES_ERR_TIMEOUT;
    default:
      if (err) *err = "poisson: register CG returned no status";
      return LES_ERR_CUDA;
  }
}

}  // namespace les
