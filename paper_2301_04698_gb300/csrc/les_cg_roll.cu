// les_cg_roll.cu -- conjugate-gradient Poisson solve in one persistent
// cooperative launch with one grid-wide reduction and one pass over memory
// per iteration (Sec. 2.4: L_c psi = b, compact 7-point Laplacian, periodic
// in x, y, mirror or periodic in z; mean of b removed, psi returned with
// zero mean).
//
// The iterates are those of standard CG.  With alpha_i and beta_i known,
// iteration i forms, for every node,
//   p_i = r_i + beta_i p_{i-1},  q_i = L_c p_i,  x += alpha_i p_i,
//   r_{i+1} = r_i - alpha_i q_i,  w = L_c r_{i+1},
// and the four sums r'.r', r'.w, r'.q, p.q (r' = r_{i+1}) in one grid-wide
// reduction.  Since p_{i+1} = r' + beta p_i and L_c is symmetric,
//   p_{i+1}.L_c p_{i+1} = r'.w + 2 beta r'.q + beta^2 p_i.q_i,
// so alpha_{i+1} = r'.r' / (that) and beta_{i+1} = r'.r' / r_i.r_i follow
// without a second reduction; every vector is still formed from its
// definition (no vector recurrence that could drift from L_c p).
//
// One pass: a 32 x 8 thread block owns a 32 x 8 column and marches a run
// of z-planes.  Planes of r_i and p_{i-1} (x / y halo of two) and of x
// (owned nodes) are copied into a shared-memory ring with cp.async several
// planes ahead of use, so the copies of a block stay in flight while it
// computes.  Per step the block forms p_i on plane k+2, q_i and r' on plane
// k+1 (halo one), and w, x and the outputs on plane k.  r and p are double-buffered by iteration parity (the
// pass reads the neighbours' r_i while writing r_{i+1}); the reduction is
// the barrier between passes.  Per iteration each node is read three times
// (r_i, p_{i-1}, x) and written three times (p_i, r_{i+1}, x).
#include <algorithm>
#include <string>

#include "les_gridsync.cuh"
#include "les_internal.h"

namespace les {
namespace {

constexpr int CX = 32, CY = 8, CH = 2;
constexpr int SX = CX + 2 * CH, SY = CY + 2 * CH, SN = SX * SY;  // staged plane with a halo of two
constexpr int D = 7;  // planes in the copy ring: the copies run up to D-3 planes ahead of use

template <typename T>
size_t roll_smem() {
  return (size_t)(2 * D * SN + D * CX * CY + 8 * SN) * sizeof(T);
}

template <typename T>
struct RollArgs {
  int nx, ny, nz, walls;
  T cx, cy, cz;  // 1/dx^2, 1/dy^2, 1/dz^2
  int ntx, nty, zrun, nchunk;
  // runs of a block as in the column CG: units u = blockIdx.x, + gridDim.x,
  // ... below nunits, then an equal share of the planes of the columns left
  int nunits, tail_planes, tail_per;
  long long n;
  const T* b;
  T* x;
  T* r[2];  // r_i in r[i & 1]
  T* p[2];  // p_i in p[i & 1]
  double* partials;
  FusedBar* bar;
  SolverCtl* ctl;
  double tol;
  int maxit;
  long long spin_cycles;
  unsigned expected;
  int guard;
};

__device__ __forceinline__ int wrapc(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}
__device__ __forceinline__ int zmapc(int k, int nz, int walls) {
  if (walls) {
    k = k < 0 ? -1 - k : (k >= nz ? 2 * nz - 1 - k : k);
    return k < 0 ? 0 : (k >= nz ? nz - 1 : k);  // planes beyond one mirror: any valid data (unused)
  }
  return wrapc(k, nz);
}
__device__ __forceinline__ int sl3(int k) { return ((k % 3) + 3) % 3; }
__device__ __forceinline__ int sl2(int k) { return ((k % 2) + 2) % 2; }
__device__ __forceinline__ int sidx(int x, int y) { return (y + CH) * SX + (x + CH); }  // x in [-2, 34)

// Long per-thread sums: FP32 within a run of 16 planes, compensated across
template <typename T>
struct LongSum;
template <>
struct LongSum<float> {
  F2 s{0.f, 0.f};
  float run = 0.f;
  __device__ __forceinline__ void add(float v) { run += v; }
  __device__ __forceinline__ void flush() {
    f2_acc(s, run);
    run = 0.f;
  }
  __device__ __forceinline__ F2 acc() const { return s; }
};
template <>
struct LongSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ double acc() const { return s; }
};

template <int NV, typename T>
__device__ __forceinline__ bool grid_long_t0(LongSum<T> (&d)[NV], GridSync& gs, double (&tot)[NV]) {
  decltype(d[0].acc()) v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    d[q].flush();
    v[q] = d[q].acc();
  }
  return grid_sum_t0<NV, 2>(v, gs, tot);  // two partials per lane in flight: within 80 registers
}

template <typename T>
__global__ void __launch_bounds__(CX* CY, 3) k_cg_roll(RollArgs<T> f) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* RAWR = reinterpret_cast<T*>(smraw);  // [D][SN] r_i as copied (halo 2)
  T* RAWP = RAWR + D * SN;                // [D][SN] p_{i-1} as copied
  T* RAWX = RAWP + D * SN;                // [D][CX * CY] x of the owned nodes
  T* PN = RAWX + D * CX * CY;             // [3][SN] p_i, planes k .. k+2
  T* QN = PN + 3 * SN;                    // [2][SN] q_i, planes k, k+1 (halo 1)
  T* RN = QN + 2 * SN;                    // [3][SN] r_{i+1}, planes k-1 .. k+1 (halo 1)
  __shared__ struct {
    T ta, tb, mean;
    int status, restart;
  } sc;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + CX * ty;
  const long long ncol = (long long)f.ntx * f.nty;
  const size_t plane = (size_t)f.nx * f.ny;
  const T cx = f.cx, cy = f.cy, cz = f.cz;
  GridSync gs{f.bar, f.partials, f.spin_cycles, f.expected, 0u};
  const long long gstride = (long long)gridDim.x * CX * CY;
  const long long gtid = (long long)blockIdx.x * CX * CY + tid;

  // compact Laplacian of a haloed plane ring at in-plane index e
  auto lap = [&](const T* lo, const T* mid, const T* hi, int e) -> T {
    const T c2 = T(2) * mid[e];
    return (mid[e - 1] + mid[e + 1] - c2) * cx + (mid[e - SX] + mid[e + SX] - c2) * cy + (lo[e] + hi[e] - c2) * cz;
  };
  // the 7-point operator straight from global memory (set-up sweeps only)
  auto lap_global = [&](const T* v, int i, int j, int k) -> T {
    const size_t row = (size_t)k * plane + (size_t)j * f.nx;
    const T c = __ldcg(v + row + i);
    const T c2 = T(2) * c;
    const T xm = __ldcg(v + row + wrapc(i - 1, f.nx)), xp = __ldcg(v + row + wrapc(i + 1, f.nx));
    const T ym = __ldcg(v + (size_t)k * plane + (size_t)wrapc(j - 1, f.ny) * f.nx + i);
    const T yp = __ldcg(v + (size_t)k * plane + (size_t)wrapc(j + 1, f.ny) * f.nx + i);
    const T zm = __ldcg(v + (size_t)zmapc(k - 1, f.nz, f.walls) * plane + (size_t)j * f.nx + i);
    const T zp = __ldcg(v + (size_t)zmapc(k + 1, f.nz, f.walls) * plane + (size_t)j * f.nx + i);
    return (xm + xp - c2) * cx + (ym + yp - c2) * cy + (zm + zp - c2) * cz;
  };
  // every node once, rows of x dealt to the blocks (one division per row, not
  // three 64-bit ones per node)
  auto each_node = [&](auto&& body) {
    const long long nrow = (long long)f.ny * f.nz;
    for (long long rw = blockIdx.x; rw < nrow; rw += gridDim.x) {
      const int j = (int)(rw % f.ny), k = (int)(rw / f.ny);
      const long long m0 = rw * f.nx;
      for (int i = tid; i < f.nx; i += CX * CY) body(m0 + i, i, j, k);
    }
  };

  double rr = 0.0, bb = 0.0, rel = 0.0, pq = 0.0;  // meaningful in thread 0
  int status = 0;  // 0 running, 1 converged, 2 maxit, 3 breakdown, 4 zero rhs, 5 timeout

  // ---- set-up: mean of b --------------------------------------------------------
  {
    LongSum<T> s[1];
    int cnt = 0;
    for (long long m = gtid; m < f.n; m += gstride) {
      s[0].add(__ldcg(f.b + m));
      if ((++cnt & 15) == 0) s[0].flush();
    }
    double t[1];
    const bool ok = grid_long_t0<1>(s, gs, t);
    if (tid == 0) {
      sc.status = ok ? 0 : 5;
      sc.mean = (T)(t[0] / (double)f.n);
    }
    __syncthreads();
    status = sc.status;
  }
  const T mean = sc.mean;
  // ---- r_0 = (b - mean) - L_c x0 into r[0]; r.r and |b - mean|^2 ----------------
  if (!status) {
    LongSum<T> s[2];
    int cnt = 0;
    each_node([&](long long m, int i, int j, int k) {
      const T bm = __ldcg(f.b + m) - mean;
      const T rv = bm - lap_global(f.x, i, j, k);
      __stcg(f.r[0] + m, rv);
      s[0].add(rv * rv);
      s[1].add(bm * bm);
      if ((++cnt & 15) == 0) {
        s[0].flush();
        s[1].flush();
      }
    });
    double t[2];
    const bool ok = grid_long_t0<2>(s, gs, t);
    if (tid == 0) {
      // the plain solver judges a learned first guess: if it leaves a larger
      // residual than x0 = 0, restart from zero (r = b - mean b, r.r = |b|^2)
      sc.status = ok ? 0 : 5;
      sc.restart = ok && f.guard && t[0] > t[1];
      rr = sc.restart ? t[1] : t[0];
      bb = t[1];
    }
    __syncthreads();
    status = sc.status;
    if (!status && sc.restart) {
      for (long long m = gtid; m < f.n; m += gstride) {
        __stcg(f.x + m, T(0));
        __stcg(f.r[0] + m, __ldcg(f.b + m) - mean);
      }
      LongSum<T> none[1];
      double t1[1];
      const bool ok2 = grid_long_t0<1>(none, gs, t1);  // a grid barrier: r_0 complete everywhere
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
  // ---- p_0 = r_0: r_0 . L_c r_0 gives alpha_0 --------------------------------------
  if (!status) {
    LongSum<T> s[1];
    int cnt = 0;
    each_node([&](long long m, int i, int j, int k) {
      s[0].add(__ldcg(f.r[0] + m) * lap_global(f.r[0], i, j, k));
      if ((++cnt & 15) == 0) s[0].flush();
    });
    double t[1];
    const bool ok = grid_long_t0<1>(s, gs, t);
    if (tid == 0) {
      pq = t[0];
      if (!ok) status = 5;
      else if (pq == 0.0 || !isfinite(pq)) status = 3;
      else {
        sc.ta = (T)(rr / pq);
        sc.tb = T(0);
      }
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
  }

  // ---- iterations ----------------------------------------------------------------
  int iter = 0;
  while (!status) {
    const T ta = sc.ta, tb = sc.tb;
    const bool first = iter == 0;
    const T* ri = f.r[iter & 1];
    T* ro = f.r[(iter + 1) & 1];
    const T* pold = f.p[(iter + 1) & 1];  // p_{i-1}
    T* pw = f.p[iter & 1];
    LongSum<T> s[4];  // r'.r', r'.w, r'.q, p.q
    int u = blockIdx.x;
    int ts = (int)blockIdx.x * f.tail_per, te = min(ts + f.tail_per, f.tail_planes);
    for (;;) {
      int col, k0, k1;
      if (u < f.nunits) {
        col = u % (int)ncol;
        k0 = (u / (int)ncol) * f.zrun;
        k1 = min(k0 + f.zrun, f.nz);
        u += gridDim.x;
      } else if (ts < te) {  // the units are whole columns here
        col = f.nunits + ts / f.nz;
        k0 = ts % f.nz;
        k1 = min(f.nz, k0 + (te - ts));
        ts += k1 - k0;
      } else {
        break;
      }
      const int x0 = (col % f.ntx) * CX, y0 = (col / f.ntx) * CY;
      const int i = x0 + tx, j = y0 + ty;
      const bool own = i < f.nx && j < f.ny;
      const int eo = sidx(tx, ty);
      // this thread's two staging slots of a plane (wrapped in-plane offsets)
      int soff[2];
      bool sok[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int e = tid + q * CX * CY;
        sok[q] = e < SN;
        const int bx = e % SX, by = e / SX;
        soff[q] = sok[q] ? wrapc(y0 - CH + by, f.ny) * f.nx + wrapc(x0 - CH + bx, f.nx) : 0;
      }
      const size_t own_off = own ? (size_t)j * f.nx + i : 0;
      // asynchronous copy of plane kk of r_i, p_{i-1} (halo 2) and x (owned
      // nodes of output planes) into ring slot kk mod D; one group per plane
      auto fetch = [&](int kk) {
        const int sl = ((kk % D) + D) % D;
        const size_t base = (size_t)zmapc(kk, f.nz, f.walls) * plane;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (!sok[q]) continue;
          const int e = tid + q * CX * CY;
          cp_async(RAWR + sl * SN + e, ri + base + soff[q]);
          if (!first) cp_async(RAWP + sl * SN + e, pold + base + soff[q]);
        }
        if (own && kk >= k0 && kk < k1) cp_async(RAWX + sl * (CX * CY) + tid, f.x + base + own_off);
        cp_commit();
      };
      auto raw = [&](const T* ring, int kk) { return ring + (((kk % D) + D) % D) * SN; };
      // p_i = r_i + beta p_{i-1} on plane kk (halo 2)
      auto place = [&](int kk) {
        const T* rr_ = raw(RAWR, kk);
        const T* pp = raw(RAWP, kk);
        T* pn = PN + sl3(kk) * SN;
        for (int e = tid; e < SN; e += CX * CY) pn[e] = first ? rr_[e] : rr_[e] + tb * pp[e];
      };
      // q_i and r_{i+1} on plane kk over the halo-one region
      auto qr = [&](int kk) {
        const T* lo = PN + sl3(kk - 1) * SN;
        const T* mid = PN + sl3(kk) * SN;
        const T* hi = PN + sl3(kk + 1) * SN;
        const T* rin = raw(RAWR, kk);
        T* qo = QN + sl2(kk) * SN;
        T* rn = RN + sl3(kk) * SN;
        for (int e1 = tid; e1 < (CX + 2) * (CY + 2); e1 += CX * CY) {
          const int e = sidx(e1 % (CX + 2) - 1, e1 / (CX + 2) - 1);
          const T qv = lap(lo, mid, hi, e);
          qo[e] = qv;
          rn[e] = rin[e] - ta * qv;
        }
      };
      // prologue: planes k0-2 .. k0+D-3 in flight; p on k0-2 .. k0+1, q and
      // r' on k0-1 and k0
      __syncthreads();  // the previous column's readers are done with the rings
      for (int kk = k0 - 2; kk <= k0 + D - 3; ++kk) fetch(kk);
      cp_wait<0>();
      __syncthreads();
      place(k0 - 2);
      place(k0 - 1);
      place(k0);
      __syncthreads();
      qr(k0 - 1);
      __syncthreads();
      place(k0 + 1);
      __syncthreads();
      qr(k0);
      int cnt = 0;
      for (int k = k0; k < k1; ++k) {
        // plane k+2 has landed (the D-5 most recent copy groups may still fly)
        cp_wait<D - 5>();
        __syncthreads();
        place(k + 2);
        __syncthreads();
        qr(k + 1);
        __syncthreads();
        if (own) {
          const size_t m = (size_t)k * plane + own_off;
          const T* rl = RN + sl3(k - 1) * SN;
          const T* rm = RN + sl3(k) * SN;
          const T* rh = RN + sl3(k + 1) * SN;
          const T rv = rm[eo];
          const T w = lap(rl, rm, rh, eo);
          const T pv = PN[sl3(k) * SN + eo];
          const T qv = QN[sl2(k) * SN + eo];
          const T xv = RAWX[(((k % D) + D) % D) * (CX * CY) + tid];
          __stcg(f.x + m, xv + ta * pv);
          __stcg(pw + m, pv);
          __stcg(ro + m, rv);
          s[0].add(rv * rv);
          s[1].add(rv * w);
          s[2].add(rv * qv);
          s[3].add(pv * qv);
        }
        if ((++cnt & 15) == 0)
#pragma unroll
          for (int q = 0; q < 4; ++q) s[q].flush();
        // the slot of plane k-2 is free: its r_i was last read by qr(k-1)
        // in the previous step and its x by its own thread
        fetch(k + D - 2);
      }
      cp_wait<0>();
    }
    double t[4];
    const bool ok = grid_long_t0<4>(s, gs, t);
    iter += 1;
    if (tid == 0) {
      if (!ok) {
        status = 5;
      } else {
        const double rr_new = t[0];
        rel = sqrt(rr_new / bb);
        if (rel <= f.tol) status = 1;
        else if (iter >= f.maxit) status = 2;
        else if (!isfinite(rr_new)) status = 3;
        else {
          const double beta = rr_new / rr;
          const double pq_new = t[1] + 2.0 * beta * t[2] + beta * beta * t[3];
          if (pq_new == 0.0 || !isfinite(pq_new)) status = 3;
          else {
            sc.ta = (T)(rr_new / pq_new);
            sc.tb = (T)beta;
          }
        }
        rr = rr_new;
      }
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
  }

  // ---- zero-mean gauge (or zero for a zero right side) ------------------------
  if (status != 5) {
    LongSum<T> s[1];
    int cnt = 0;
    for (long long m = gtid; m < f.n; m += gstride) {
      s[0].add(__ldcg(f.x + m));
      if ((++cnt & 15) == 0) s[0].flush();
    }
    double t[1];
    const bool ok = grid_long_t0<1>(s, gs, t);
    if (tid == 0) {
      if (!ok) status = 5;
      sc.mean = (T)(t[0] / (double)f.n);
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
    if (status != 5) {
      const T mx = sc.mean;
      for (long long m = gtid; m < f.n; m += gstride) __stcg(f.x + m, status == 4 ? T(0) : __ldcg(f.x + m) - mx);
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    f.ctl->iter = iter;
    f.ctl->rel = rel;
    f.ctl->done = status;
  }
}

}  // namespace

template <typename T>
int poisson_solve_roll(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit,
                       int* iters, double* rel, std::string* err) {
  RollArgs<T> f;
  f.nx = a.g.nx;
  f.ny = a.g.ny;
  f.nz = a.g.nz;
  f.walls = a.g.walls;
  f.cx = a.g.idx * a.g.idx;
  f.cy = a.g.idy * a.g.idy;
  f.cz = a.g.idz * a.g.idz;
  f.ntx = (f.nx + CX - 1) / CX;
  f.nty = (f.ny + CY - 1) / CY;
  f.n = (long long)f.nx * f.ny * f.nz;
  f.b = b;
  f.x = x;
  f.r[0] = a.r;
  f.r[1] = a.q;
  f.p[0] = a.p0;
  f.p[1] = a.p1;
  f.partials = a.partials;
  f.bar = a.bar;
  f.ctl = a.ctl;
  f.tol = tol;
  f.maxit = maxit;
  f.spin_cycles = fc.spin_cycles;
  f.guard = a.guard;
  int per_sm = 0, dev = 0, nsm = 0;
  cudaError_t e;
  const void* kern = (const void*)k_cg_roll<T>;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)roll_smem<T>())) !=
          cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CX * CY, roll_smem<T>())) != cudaSuccess) {
    if (err) *err = std::string("rolling CG occupancy: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  long long G = (long long)std::max(1, per_sm) * nsm;
  G = std::min<long long>(G, fc.max_blocks);
  G = std::min<long long>(G, 8LL * nsm);  // the partials hold 2 x kSumSlot words of 8 blocks per SM
  // z-runs as long as possible (each run re-forms two planes of p and one of
  // q, r' below it), dealt to the G persistent blocks as in the column CG:
  // fewer columns than blocks, at most G units (one turn); more, whole
  // columns in full turns and the columns left in equal plane shares
  const long long ncol = (long long)f.ntx * f.nty;
  if (ncol >= G) {
    f.zrun = f.nz;
    f.nchunk = 1;
    f.nunits = (int)((ncol / G) * G);
    f.tail_planes = (int)((ncol - f.nunits) * f.nz);
    f.tail_per = (int)((f.tail_planes + G - 1) / G);
  } else {
    const long long want = std::max<long long>(1, std::min<long long>((long long)f.nz, G / ncol));
    f.zrun = (int)((f.nz + want - 1) / want);
    f.nchunk = (f.nz + f.zrun - 1) / f.zrun;
    f.nunits = (int)(ncol * f.nchunk);
    f.tail_planes = 0;
    f.tail_per = 0;
    G = std::max<long long>(1, std::min<long long>(G, f.nunits));
  }
  f.expected = (unsigned)G + (unsigned)std::max(0, fc.missing);
  if ((e = cudaMemsetAsync(a.bar, 0, sizeof(FusedBar), a.st)) != cudaSuccess) {
    if (err) *err = std::string("rolling CG barrier reset: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  void* args[] = {&f};
  {
    ProfScope ps(a.prof, KI_CG_ROLL, a.st);
    e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), dim3(CX, CY), args, roll_smem<T>(), a.st);
  }
  if (e != cudaSuccess) {
    if (err) *err = std::string("rolling CG launch: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  if ((e = cudaMemcpyAsync(a.ctl_host, a.ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, a.st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(a.st)) != cudaSuccess) {
    if (err) *err = std::string("rolling CG: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  const SolverCtl& c = *a.ctl_host;
  if (iters) *iters = c.iter;
  if (rel) *rel = c.rel;
  // algorithmic traffic of the solve (kCgIterFields per iteration; this
  // kernel streams 6: r, p_old, x in; p, r, x out; plus one set-up sweep
  // for alpha_0)
  if (a.prof) a.prof->bytes[KI_CG_ROLL] += (kCgSetupFields + 1.0 + kCgIterFields * c.iter) * (double)f.n * sizeof(T);
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
      if (err) *err = "poisson: rolling solver returned no status";
      return LES_ERR_CUDA;
  }
}

template int poisson_solve_roll<float>(const SolverArgs<float>&, const FusedCfg&, const float*, float*, double, int,
                                       int*, double*, std::string*);
template int poisson_solve_roll<double>(const SolverArgs<double>&, const FusedCfg&, const double*, double*, double,
                                        int, int*, double*, std::string*);

}  // namespace les
