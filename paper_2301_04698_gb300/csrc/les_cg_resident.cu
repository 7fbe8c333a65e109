// les_cg_resident.cu -- the conjugate-gradient Poisson solve with its
// vectors resident in shared memory (Sec. 2.4: L_c psi = b, compact 7-point
// Laplacian, periodic in x, y, mirror or periodic in z; mean of b removed,
// psi returned with zero mean).
//
// When the whole grid fits in the GPU's shared memory (a 128 x 128 x 96 FP32
// grid needs about 31 MB of the 34 MB on 152 SMs), every iteration of the
// streaming solver is dominated by the latency of its passes through L2, not
// by their bytes.  Here each block of one persistent cooperative launch owns
// a brick of bx x by x bz nodes for the whole solve and keeps x, r, p (with a
// one-node ghost layer), q = L_c p and r at the ghost nodes in shared memory.
// An iteration is two passes over the brick and one grid-wide sum:
//   matvec   q = L_c p, q faces published; p.q, r.r, r.q and q.q
//   (grid-wide sum: alpha, and beta from |r - alpha q|^2 expanded in the
//   four sums, so that no second sum is needed for r_{i+1}.r_{i+1})
//   update   x += alpha p, r -= alpha q, p = r + beta p; at the ghost nodes
//            r -= alpha q with the neighbours' published q faces, then
//            p = r + beta p
// The only global traffic is the exchange of q faces (double-buffered by
// parity) and the first residual's faces.  The grid sum (les_gridsync.cuh)
// accumulates FP32 dot products as compensated FP32 pairs, FP64 ones in
// FP64.  Ghost loads are issued in one batch whose latency overlaps the
// owned update.
#include <algorithm>
#include <string>

#include "les_gridsync.cuh"
#include "les_internal.h"

namespace les {
namespace {

constexpr int kResThreads = 512;

template <typename T>
struct ResArgs {
  int nx, ny, nz, walls;
  T cx, cy, cz;      // 1/dx^2, 1/dy^2, 1/dz^2
  int by;            // brick extent in y (x extent: the template BX)
  int px, py, pz;    // bricks along x, y and z (z extents differ by at most one)
  long long n;
  const T* b;
  T* x;
  T* rg;             // published faces of the first residual
  T* qg0;            // published faces of q = L_c p, even iterations
  T* qg1;            // ... odd iterations
  double* partials;  // two slots of kSumSlot words per block
  FusedBar* bar;
  SolverCtl* ctl;
  double tol;
  int maxit;
  long long spin_cycles;
  unsigned expected;
  int guard;
};

__device__ __forceinline__ int zghost(int k, int nz, int walls) {
  if (walls) return k < 0 ? -1 - k : (k >= nz ? 2 * nz - 1 - k : k);
  return k < 0 ? k + nz : (k >= nz ? k - nz : k);
}

template <typename T, int BX>
__global__ void __launch_bounds__(kResThreads, 1) k_cg_resident(ResArgs<T> f) {
  constexpr int L = BX / 32;  // nodes per lane along a brick row
  // ghost rows per warp (and x-face ghosts per thread) whose loads are in
  // flight together, within the registers
  constexpr int RB = sizeof(T) == 4 ? (L >= 4 ? 3 : 4) : (L >= 2 ? 1 : 2);
  constexpr int XB = sizeof(T) == 4 ? 4 : 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  const int bi = blockIdx.x % f.px, bj = (blockIdx.x / f.px) % f.py, bk = blockIdx.x / (f.px * f.py);
  // z extents: the first nz mod pz bricks hold one plane more
  const int zbase = f.nz / f.pz, zrem = f.nz % f.pz;
  const int by = f.by, bz = zbase + (bk < zrem ? 1 : 0);
  const int i0 = bi * BX, j0 = bj * by, k0 = bk * zbase + min(bk, zrem);
  const int SY = BX + 2, SZ = (BX + 2) * (by + 2);  // strides of the haloed p brick
  const int nrow = by * bz;
  const int bcells = BX * nrow;
  // A brick spanning the periodic x extent is its own x neighbour: its x
  // ghosts are copies of its own end nodes, written with them, and its x
  // faces are not published.
  const bool xself = f.px == 1;
  const int nr = 2 * by + 2 * bz;          // ghost rows along x (z faces, then y faces)
  const int nxg = xself ? 0 : 2 * nrow;    // strided x-face ghosts
  T* P = reinterpret_cast<T*>(smraw);      // (BX + 2)(by + 2)(bz + 2): p with its ghost layer
  T* R = P + SZ * (bz + 2);                // BX by bz
  T* X = R + bcells;                       // BX by bz
  T* Q = X + bcells;                       // BX by bz: L_c p of this iteration
  T* RG = Q + bcells;                      // r at the ghost nodes: nr BX rows, then nxg x-face nodes
  // per brick row: P offset | face bit, global offset (8-byte aligned: the
  // T arrays above hold an even number of elements)
  int2* ROWS = reinterpret_cast<int2*>(RG + nr * BX + nxg);
  const T cx = f.cx, cy = f.cy, cz = f.cz;

  // global index of local node (lx, ly, lz), at most one node outside the brick
  auto gidx = [&](int lx, int ly, int lz) -> size_t {
    int i = i0 + lx, j = j0 + ly;
    i = i < 0 ? i + f.nx : (i >= f.nx ? i - f.nx : i);
    j = j < 0 ? j + f.ny : (j >= f.ny ? j - f.ny : j);
    const int k = zghost(k0 + lz, f.nz, f.walls);
    return ((size_t)k * f.ny + j) * f.nx + i;
  };
  // second differences formed before scaling: for smooth p they are small
  // differences of nearly equal values, exact in floating point
  auto Lc = [&](int pi) -> T {
    const T c2 = T(2) * P[pi];
    return (P[pi - 1] + P[pi + 1] - c2) * cx + (P[pi - SY] + P[pi + SY] - c2) * cy +
           (P[pi - SZ] + P[pi + SZ] - c2) * cz;
  };
  // the row table: row index arithmetic once per launch, not once per pass.
  // Surface rows come first, so that the face stores of a pass are issued
  // early and have landed by the grid sum's release at its end.
  const size_t gbase = ((size_t)k0 * f.ny + j0) * f.nx + i0;
  {
    const int by2 = max(by - 2, 0), bz2 = max(bz - 2, 0);
    const int nface = nrow - by2 * bz2;
    for (int row = tid; row < nrow; row += nthr) {
      const int ly = row % by, lz = row / by;
      const bool zin = lz >= 1 && lz <= bz - 2;
      const bool rface = !(zin && ly >= 1 && ly <= by - 2);
      // interior rows before this one in (ly, lz) order
      const int before = min(max(lz - 1, 0), bz2) * by2 + (zin ? min(max(ly - 1, 0), by2) : 0);
      const int pos = rface ? row - before : nface + before;
      const int prow = (lz + 1) * SZ + (ly + 1) * SY + 1;
      ROWS[pos] = make_int2(prow | (rface ? (int)0x80000000u : 0), (lz * f.ny + ly) * f.nx);
    }
  }
  __syncthreads();
  // store p at owned node (c, pi), and at its periodic x image in the ghost
  // layer for a brick that is its own x neighbour
  auto put_p = [&](int c, int pi, T v) {
    P[pi] = v;
    if (xself) {
      const int lx = c & (BX - 1);
      if (lx == 0) P[pi + BX] = v;
      else if (lx == BX - 1) P[pi - BX] = v;
    }
  };
  // body(c, pi, g, face) for every owned node: c its index in R / X / Q, pi in
  // P, g in global memory; face: the node lies on a brick surface that a
  // neighbour reads
  auto own = [&](auto&& body) {
    for (int row = warp; row < nrow; row += nwarp) {
      const int2 t = ROWS[row];
      const bool rface = t.x < 0;
      const int prow = t.x & 0x7fffffff;
      const size_t grow = gbase + (unsigned)t.y;
#pragma unroll
      for (int u = 0; u < L; ++u) {
        const int lx = lane + 32 * u;
        body(row * BX + lx, prow + lx, grow + lx, rface || (!xself && (lx == 0 || lx == BX - 1)));
      }
    }
  };
  // body(c0, prow, grow, rface) for every owned row: the row's nodes are
  // c0 + lx in R / X / Q, prow + lx in P and grow + lx in global memory.  The
  // passes of the iteration handle a row's L nodes per lane together, with
  // every shared-memory load issued before the first store (the compiler
  // cannot reorder them across stores to the other arrays of the block).
  auto own_rows = [&](auto&& body) {
    for (int row = warp; row < nrow; row += nwarp) {
      const int2 t = ROWS[row];
      body(row * BX, t.x & 0x7fffffff, gbase + (unsigned)t.y, t.x < 0);
    }
  };
  // For each face-neighbour node outside the brick (edges and corners are
  // not used by the 7-point stencil) load a = A at its global node and call
  // put(pi, k, a) with its index pi in P and k in RG.  Every load of a batch
  // is issued before any loaded value is used, so a batch costs one round of
  // memory latency; when one batch per thread covers all ghosts, between()
  // runs while the loads are in flight.
  const bool one_round = nr <= RB * nwarp && nxg <= XB * nthr;
  auto ghost_row = [&](int row, int& ly, int& lz) {
    if (row < 2 * by) {
      ly = row >> 1;
      lz = (row & 1) ? bz : -1;
    } else {
      lz = (row - 2 * by) >> 1;
      ly = (row & 1) ? by : -1;
    }
  };
  auto xghost = [&](int c, int& ly, int& lz, int& lx) {
    const int row = c >> 1;
    ly = row % by;
    lz = row / by;
    lx = (c & 1) ? BX : -1;
  };
  auto ghosts = [&](const T* A, auto&& between, auto&& put) {
    if (one_round) {
      T va[RB][L], xa[XB];
      int pr[RB], xpi[XB];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int row = warp + q * nwarp;
        pr[q] = -1;
        if (row < nr) {
          int ly, lz;
          ghost_row(row, ly, lz);
          pr[q] = (lz + 1) * SZ + (ly + 1) * SY + 1;
          const size_t g0 = gidx(0, ly, lz);
#pragma unroll
          for (int u = 0; u < L; ++u) va[q][u] = __ldcg(A + g0 + lane + 32 * u);
        }
      }
#pragma unroll
      for (int q = 0; q < XB; ++q) {
        const int c = tid + q * nthr;
        xpi[q] = -1;
        if (c < nxg) {
          int ly, lz, lx;
          xghost(c, ly, lz, lx);
          xpi[q] = (lz + 1) * SZ + (ly + 1) * SY + 1 + lx;
          xa[q] = __ldcg(A + gidx(lx, ly, lz));
        }
      }
      between();
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (pr[q] >= 0)
#pragma unroll
          for (int u = 0; u < L; ++u) put(pr[q] + lane + 32 * u, (warp + q * nwarp) * BX + lane + 32 * u, va[q][u]);
#pragma unroll
      for (int q = 0; q < XB; ++q)
        if (xpi[q] >= 0) put(xpi[q], nr * BX + tid + q * nthr, xa[q]);
      return;
    }
    between();
    for (int r0 = warp; r0 < nr; r0 += RB * nwarp) {
      T va[RB][L];
      int pr[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int row = r0 + q * nwarp;
        pr[q] = -1;
        if (row < nr) {
          int ly, lz;
          ghost_row(row, ly, lz);
          pr[q] = (lz + 1) * SZ + (ly + 1) * SY + 1;
          const size_t g0 = gidx(0, ly, lz);
#pragma unroll
          for (int u = 0; u < L; ++u) va[q][u] = __ldcg(A + g0 + lane + 32 * u);
        }
      }
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (pr[q] >= 0)
#pragma unroll
          for (int u = 0; u < L; ++u) put(pr[q] + lane + 32 * u, (r0 + q * nwarp) * BX + lane + 32 * u, va[q][u]);
    }
    for (int c0 = tid; c0 < nxg; c0 += XB * nthr) {
      T xa[XB];
      int pi[XB];
#pragma unroll
      for (int q = 0; q < XB; ++q) {
        const int c = c0 + q * nthr;
        pi[q] = -1;
        if (c < nxg) {
          int ly, lz, lx;
          xghost(c, ly, lz, lx);
          pi[q] = (lz + 1) * SZ + (ly + 1) * SY + 1 + lx;
          xa[q] = __ldcg(A + gidx(lx, ly, lz));
        }
      }
#pragma unroll
      for (int q = 0; q < XB; ++q)
        if (pi[q] >= 0) put(pi[q], nr * BX + c0 + q * nthr, xa[q]);
    }
  };
  auto nothing = [] {};

  GridSync gs{f.bar, f.partials, f.spin_cycles, f.expected, 0u};
  // The scalar recurrences of CG run in thread 0 (FP64 division and square
  // root are long instruction sequences on this GPU); thread 0 broadcasts
  // the status and the FP32/FP64 coefficients through shared memory.
  __shared__ struct {
    T ta, tb, mean;
    int status, restart;
  } sc;
  double rr = 0.0, bb = 0.0, rel = 0.0;  // meaningful in thread 0
  int status = 0;  // 0 running, 1 converged, 2 maxit, 3 breakdown, 4 zero rhs, 5 timeout
  // mean of b; b staged in R
  {
    Dot<T> a1[1];
    own([&](int c, int, size_t g, bool) {
      const T v = __ldcg(f.b + g);
      R[c] = v;
      a1[0].add(v);
    });
    double t[1];
    const bool ok = grid_dot_t0<1>(a1, gs, t);
    if (tid == 0) {
      sc.status = ok ? 0 : 5;
      sc.mean = (T)(t[0] / (double)f.n);
    }
    __syncthreads();
    status = sc.status;
  }
  const T mean = sc.mean;

  // x0 with its ghosts; r = (b - mean) - L_c x0, published; r.r and |b - mean|^2
  if (!status) {
    own([&](int c, int pi, size_t g, bool) {
      const T v = __ldcg(f.x + g);
      X[c] = v;
      put_p(c, pi, v);
    });
    ghosts(f.x, nothing, [&](int pi, int, T v) { P[pi] = v; });
    __syncthreads();
    Dot<T> a2[2];
    own([&](int c, int pi, size_t g, bool face) {
      const T bm = R[c] - mean;
      const T rv = bm - Lc(pi);
      R[c] = rv;
      if (face) __stcg(f.rg + g, rv);
      a2[0].add(rv * rv);
      a2[1].add(bm * bm);
    });
    double s2[2];
    const bool ok = grid_dot_t0<2>(a2, gs, s2);
    if (tid == 0) {
      // the plain solver judges a learned first guess: if it leaves a larger
      // residual than x0 = 0, restart from zero (r = b - mean b, r.r = |b|^2)
      sc.status = ok ? 0 : 5;
      sc.restart = ok && f.guard && s2[0] > s2[1];
      rr = sc.restart ? s2[1] : s2[0];
      bb = s2[1];
    }
    __syncthreads();
    status = sc.status;
    if (!status && sc.restart) {
      own([&](int c, int, size_t g, bool face) {
        const T rv = __ldcg(f.b + g) - mean;
        X[c] = T(0);
        R[c] = rv;
        if (face) __stcg(f.rg + g, rv);
      });
      Dot<T> none[1];
      double t[1];
      const bool ok2 = grid_dot_t0<1>(none, gs, t);  // a grid barrier: the new faces are visible
      if (tid == 0) sc.status = ok2 ? 0 : 5;
      __syncthreads();
      status = sc.status;
    }
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

  // The iterations, one grid-wide sum each.  With r = r_i, p = p_i and
  // q = L_c p_i, the sum yields p.q, r.r, r.q and q.q; then
  //   alpha = r.r / p.q,   |r_{i+1}|^2 = r.r - 2 alpha r.q + alpha^2 q.q,
  //   beta = |r_{i+1}|^2 / r.r,
  // and one pass forms x += alpha p, r_{i+1} = r - alpha q and
  // p_{i+1} = r_{i+1} + beta p.  The neighbours' r enters through the ghost
  // layer: each brick keeps r at its ghost nodes and updates it with the q
  // faces its neighbours published before the sum, so no second exchange is
  // needed.  Convergence is judged on the r.r of each sum (the residual of
  // the current x) as r.r <= tol^2 |b - mean|^2, in the sums' precision.
  using Acc = decltype(Dot<T>().acc());   // FP32 pair (FP32 solve) or FP64
  Acc rr_stop, rr_last;                   // meaningful in thread 0
  acc_from(f.tol * f.tol * bb, rr_stop);  // compared in the totals' own precision
  acc_from(rr, rr_last);
  int iter = 0;
  // alpha and beta from the totals (p.q, r.r, r.q, q.q); false on a zero or
  // non-finite p.q or r.r.  An FP32 solve takes them in FP32 from the high
  // parts of the compensated totals: those carry the dot products' own
  // precision, and the chain of FP64 operations through one thread would
  // cost about a microsecond per iteration on this GPU.
  auto scalars = [&](const auto(&t)[4], T& ta, T& tb) -> bool {
    if constexpr (sizeof(T) == 4) {
      const float pq = t[0].hi, r2 = t[1].hi, rq = t[2].hi, q2 = t[3].hi;
      if (!(pq != 0.f) || !isfinite(pq) || !isfinite(r2)) return false;
      const float alpha = r2 / pq;
      const float rn = fmaf(alpha * alpha, q2, fmaf(-2.f * alpha, rq, r2));  // |r - alpha q|^2
      ta = alpha;
      tb = rn / r2;
    } else {
      const double pq = t[0], r2 = t[1], rq = t[2], q2 = t[3];
      if (!(pq != 0.0) || !isfinite(pq) || !isfinite(r2)) return false;
      const double inv = 1.0 / (r2 * pq);  // one FP64 division for both
      const double alpha = r2 * r2 * inv;
      const double rn = fma(alpha * alpha, q2, fma(-2.0 * alpha, rq, r2));
      ta = alpha;
      tb = rn * (pq * inv);
    }
    return true;
  };
  if (!status) {
    // p_0 = r_0 with the ghosts of r_0
    ghosts(
        f.rg,
        [&] { own([&](int c, int pi, size_t, bool) { put_p(c, pi, R[c]); }); },
        [&](int pi, int k, T v) {
          RG[k] = v;
          P[pi] = v;
        });
    __syncthreads();
    for (;;) {
      T* qw = (iter & 1) ? f.qg1 : f.qg0;  // this iteration's q faces
      Dot<T> d[4];                         // p.q, r.r, r.q, q.q
      own_rows([&](int c0, int prow, size_t grow, bool rface) {
        T pc[L], pw[L], pe[L], ps[L], pn[L], pd[L], pu[L], rv[L];
#pragma unroll
        for (int u = 0; u < L; ++u) {
          const int pi = prow + lane + 32 * u;
          pc[u] = P[pi];
          pw[u] = P[pi - 1];
          pe[u] = P[pi + 1];
          ps[u] = P[pi - SY];
          pn[u] = P[pi + SY];
          pd[u] = P[pi - SZ];
          pu[u] = P[pi + SZ];
          rv[u] = R[c0 + lane + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < L; ++u) {
          const int lx = lane + 32 * u;
          const T c2 = T(2) * pc[u];
          const T qv = (pw[u] + pe[u] - c2) * cx + (ps[u] + pn[u] - c2) * cy + (pd[u] + pu[u] - c2) * cz;
          Q[c0 + lx] = qv;
          if (rface || (!xself && (lx == 0 || lx == BX - 1))) __stcg(qw + grow + lx, qv);
          d[0].add(pc[u] * qv);
          d[1].add(rv[u] * rv[u]);
          d[2].add(rv[u] * qv);
          d[3].add(qv * qv);
        }
      });
      Acc v[4], t[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = d[q].acc();
      const bool ok = grid_sum_t0_acc<4>(v, gs, t, NoWork{});
      // the sum has completed (or timed out): from here every thread may read
      // the q faces the other blocks published before it
      __syncthreads();
      // the update pass.  The loads of the neighbours' q faces are issued
      // first; while they are in flight thread 0 forms alpha, beta and the
      // status, then the owned nodes are updated.
      T ta = T(0), tb = T(0);
      ghosts(
          qw,
          [&] {
            if (tid == 0) {
              if (!ok) {
                status = 5;
              } else {
                rr_last = t[1];
                if (acc_le(t[1], rr_stop)) status = 1;
                else if (iter >= f.maxit) status = 2;
                else if (!scalars(t, sc.ta, sc.tb)) status = 3;
              }
              sc.status = status;
            }
            __syncthreads();
            status = sc.status;
            if (status) return;
            ta = sc.ta;
            tb = sc.tb;
            own_rows([&](int c0, int prow, size_t, bool) {
              T pv[L], xv[L], rv[L], qv[L];
#pragma unroll
              for (int u = 0; u < L; ++u) {
                const int lx = lane + 32 * u;
                pv[u] = P[prow + lx];
                xv[u] = X[c0 + lx];
                rv[u] = R[c0 + lx];
                qv[u] = Q[c0 + lx];
              }
#pragma unroll
              for (int u = 0; u < L; ++u) {
                const int lx = lane + 32 * u;
                X[c0 + lx] = xv[u] + ta * pv[u];
                const T r1 = rv[u] - ta * qv[u];
                R[c0 + lx] = r1;
                put_p(c0 + lx, prow + lx, r1 + tb * pv[u]);
              }
            });
          },
          [&](int pi, int k, T qv) {
            const T rv = RG[k] - ta * qv;
            RG[k] = rv;
            P[pi] = rv + tb * P[pi];
          });
      if (status) break;  // the ghosts just written are not used
      iter += 1;
      __syncthreads();
    }
  }
  if (tid == 0 && iter > 0 && bb > 0.0) {
    rr = acc_value(rr_last);
    rel = sqrt(rr / bb);
  }

  // zero-mean gauge (or zero for a zero right side), written back to x
  if (status != 5) {
    Dot<T> ax[1];
    own([&](int c, int, size_t, bool) { ax[0].add(X[c]); });
    double t[1];
    const bool ok = grid_dot_t0<1>(ax, gs, t);
    if (tid == 0) {
      if (!ok) status = 5;
      sc.mean = (T)(t[0] / (double)f.n);
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
    if (status != 5) {
      const T mx = sc.mean;
      own([&](int c, int, size_t g, bool) { __stcg(f.x + g, status == 4 ? T(0) : X[c] - mx); });
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    f.ctl->iter = iter;
    f.ctl->rel = rel;
    f.ctl->done = status;
  }
}

struct Plan {
  int bx = 0, by = 0, bz = 0, px = 0, py = 0, pz = 0;  // bz: the largest brick extent in z
  size_t smem = 0;
};

template <typename T>
size_t resident_smem(int bx, int by, int bz, bool xself) {
  const size_t ghosts = (size_t)(2 * by + 2 * bz) * bx + (xself ? 0 : 2 * (size_t)by * bz);
  return ((size_t)(bx + 2) * (by + 2) * (bz + 2) + 3 * (size_t)bx * by * bz + ghosts) * sizeof(T) +
         (size_t)by * bz * sizeof(int2);
}

// Brick decomposition: bx in {128, 64, 32} dividing nx, by | ny, pz bricks
// along z of nz / pz planes (rounded up or down), at most one brick per SM and
// within the per-block shared memory; among those the one with the least
// work for its largest brick (owned nodes + ghost nodes + a per-block
// barrier cost).
template <typename T>
bool make_plan(const Grid<T>& g, int nsm, size_t smem_max, int max_blocks, Plan& best) {
  long long best_score = -1;
  const int gmax = std::min(nsm, max_blocks);
  for (int bx : {128, 64, 32}) {
    if (g.nx % bx) continue;
    const bool xself = bx == g.nx;
    for (int by = 1; by <= g.ny; ++by) {
      if (g.ny % by) continue;
      for (int pz = 1; pz <= g.nz; ++pz) {
        const int bz = (g.nz + pz - 1) / pz;
        if (pz > 1 && (g.nz + pz - 2) / (pz - 1) == bz) continue;  // as large, with more bricks
        const long long G = (long long)(g.nx / bx) * (g.ny / by) * pz;
        if (G > gmax) break;
        const size_t smem = resident_smem<T>(bx, by, bz, xself);
        if (smem > smem_max) continue;
        const long long cells = (long long)bx * by * bz;
        // x-face ghosts are strided single nodes, one 32-byte sector each:
        // weighted as eight; a brick as wide as the grid loads none
        const long long ghosts = 2LL * bx * by + 2LL * bx * bz + (xself ? 0LL : 16LL * by * bz);
        const long long score = cells + ghosts + 4 * G;
        if (best_score < 0 || score < best_score) {
          best_score = score;
          best.bx = bx;
          best.by = by;
          best.bz = bz;
          best.px = g.nx / bx;
          best.py = g.ny / by;
          best.pz = pz;
          best.smem = smem;
        }
      }
    }
  }
  return best_score >= 0;
}

template <typename T>
const void* resident_kernel(int bx) {
  switch (bx) {
    case 128: return (const void*)k_cg_resident<T, 128>;
    case 64: return (const void*)k_cg_resident<T, 64>;
    case 32: return (const void*)k_cg_resident<T, 32>;
    default: return nullptr;
  }
}

}  // namespace

template <typename T>
int poisson_solve_resident(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit,
                           int* iters, double* rel, std::string* err, bool* used) {
  *used = false;
  if (!(a.op == LES_OP_COMPACT && a.solver == LES_SOLVER_CG && a.g.nz >= 2 && a.bar && a.r && a.p0 && a.p1))
    return LES_OK;
  // FP32 grids 128 nodes wide: p, r and q in registers (les_cg_regs.cu)
  if constexpr (sizeof(T) == 4) {
    if (fc.resident == 0) {
      const int rc = poisson_solve_regs(a, fc, b, x, tol, maxit, iters, rel, err, used);
      if (*used || rc != LES_OK) return rc;
    }
  }
  int dev = 0, nsm = 0, smem_optin = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) {
    if (err) *err = std::string("resident CG: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  Plan pl;
  // leave room for the reductions' static shared memory (about 2 KB)
  if (!make_plan(a.g, nsm, (size_t)std::max(0, smem_optin - 3072), fc.max_blocks, pl)) return LES_OK;
  const void* kern = resident_kernel<T>(pl.bx);
  int per_sm = 0;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kResThreads, pl.smem)) != cudaSuccess) {
    if (err) *err = std::string("resident CG occupancy: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  const long long G = (long long)pl.px * pl.py * pl.pz;
  if (per_sm < 1 || G > (long long)per_sm * nsm) return LES_OK;  // not co-resident: stream instead
  ResArgs<T> f;
  f.nx = a.g.nx;
  f.ny = a.g.ny;
  f.nz = a.g.nz;
  f.walls = a.g.walls;
  f.cx = a.g.idx * a.g.idx;
  f.cy = a.g.idy * a.g.idy;
  f.cz = a.g.idz * a.g.idz;
  f.by = pl.by;
  f.px = pl.px;
  f.py = pl.py;
  f.pz = pl.pz;
  f.n = (long long)f.nx * f.ny * f.nz;
  f.b = b;
  f.x = x;
  f.rg = a.r;
  f.qg0 = a.p0;
  f.qg1 = a.p1;
  f.partials = a.partials;
  f.bar = a.bar;
  f.ctl = a.ctl;
  f.tol = tol;
  f.maxit = maxit;
  f.spin_cycles = fc.spin_cycles;
  f.expected = (unsigned)G + (unsigned)std::max(0, fc.missing);
  f.guard = a.guard;
  *used = true;
  if ((e = cudaMemsetAsync(a.bar, 0, sizeof(FusedBar), a.st)) != cudaSuccess) {
    if (err) *err = std::string("resident CG barrier reset: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  void* args[] = {&f};
  {
    ProfScope ps(a.prof, KI_CG_RESIDENT, a.st);
    e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), dim3(kResThreads), args, pl.smem, a.st);
  }
  if (e != cudaSuccess) {
    if (err) *err = std::string("resident CG launch: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  if ((e = cudaMemcpyAsync(a.ctl_host, a.ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, a.st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(a.st)) != cudaSuccess) {
    if (err) *err = std::string("resident CG: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  const SolverCtl& c = *a.ctl_host;
  if (iters) *iters = c.iter;
  if (rel) *rel = c.rel;
  // algorithmic traffic of the solve (kCgIterFields per iteration), so that
  // every CG kernel reports a comparable rate; this one keeps its vectors
  // on chip and moves only b, x and the brick faces through DRAM
  if (a.prof) a.prof->bytes[KI_CG_RESIDENT] += (kCgSetupFields + kCgIterFields * c.iter) * (double)f.n * sizeof(T);
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
      if (err) *err = "poisson: resident solver returned no status";
      return LES_ERR_CUDA;
  }
}

template int poisson_solve_resident<float>(const SolverArgs<float>&, const FusedCfg&, const float*, float*, double,
                                           int, int*, double*, std::string*, bool*);
template int poisson_solve_resident<double>(const SolverArgs<double>&, const FusedCfg&, const double*, double*,
                                            double, int, int*, double*, std::string*, bool*);

}  // namespace les
