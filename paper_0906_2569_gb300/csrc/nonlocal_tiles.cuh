// Tile functions of the float64 nonlocal term (paper Sec. 3: becp = <beta|psi>, w = D becp,
// hpsi += beta w) shared by the one-launch-per-kernel forms (nonlocal_fp64.cu) and the persistent
// batched H|psi> (local_fast.cu): each call does one CTA's tile; the callers map their blocks onto
// tiles.  Included inside an anonymous namespace of namespace hpsi, once per translation unit.
#pragma once

// acc += conj(x) y and acc += x y, four float64 FMAs each
__device__ __forceinline__ void cmac_conj(double2& acc, double2 x, double2 y) {
  acc.x = fma(x.x, y.x, acc.x);
  acc.x = fma(x.y, y.y, acc.x);
  acc.y = fma(x.x, y.y, acc.y);
  acc.y = fma(-x.y, y.x, acc.y);
}
__device__ __forceinline__ void cmac(double2& acc, double2 x, double2 y) {
  acc.x = fma(x.x, y.x, acc.x);
  acc.x = fma(-x.y, y.y, acc.x);
  acc.y = fma(x.x, y.y, acc.y);
  acc.y = fma(x.y, y.x, acc.y);
}

constexpr int CB_TP = 32;   // projectors per CTA
constexpr int CB_TB = 32;   // bands per CTA
constexpr int CB_TK = 32;   // G per shared-memory tile

constexpr int CB_SMEM = (CB_TP + CB_TB) * (CB_TK + 1);   // double2 entries of shared memory

// part[split][b][p] = sum_{G in split} conj(beta[p][G]) psi[b][G] for the TP projectors of tile tp
// and the CB_TB bands of tile tb; sm: CB_SMEM entries of shared memory.  TP = 32: 2 x 2 outputs per
// thread; TP = 16 and 8 (items with few projectors): 1 x 2 and 1 x 1, so that fewer rows of the
// tile are padding.  Each output is the same chain of FMAs over G in order whatever TP is.
template <int TP>
__device__ __forceinline__ void calbec_tile_t(int npw, int nproj, int nb, int kchunk, const double2* __restrict__ beta,
                                              const double2* __restrict__ psi, double2* __restrict__ part, int tp,
                                              int tb, int split, double2* sm) {
  constexpr int TX = TP < 16 ? TP : 16;        // threads along the projectors
  constexpr int TY = 256 / TX;                 // threads along the bands
  constexpr int PI = TP / TX, BJ = CB_TB / TY; // outputs per thread
  static_assert(TP <= CB_TP && PI >= 1 && BJ >= 1 && TX * TY == 256, "calbec tile shape");
  auto sb = reinterpret_cast<double2 (*)[CB_TK + 1]>(sm);                    // [TP][CB_TK + 1]
  auto sp = reinterpret_cast<double2 (*)[CB_TK + 1]>(sm + TP * (CB_TK + 1));  // [CB_TB][CB_TK + 1]
  const int p0 = tp * TP, b0 = tb * CB_TB;
  const int gbeg = split * kchunk, gend = min(npw, gbeg + kchunk);
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;   // tx -> p, ty -> b
  double2 acc[PI][BJ];
#pragma unroll
  for (int i = 0; i < PI; ++i)
#pragma unroll
    for (int j = 0; j < BJ; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int g0 = gbeg; g0 < gend; g0 += CB_TK) {
    for (int i = threadIdx.x; i < TP * CB_TK; i += 256) {
      const int r = i / CB_TK, cc = i % CB_TK;
      const int g = g0 + cc;
      sb[r][cc] = (p0 + r < nproj && g < gend) ? beta[(size_t)(p0 + r) * npw + g] : make_double2(0.0, 0.0);
    }
    for (int i = threadIdx.x; i < CB_TB * CB_TK; i += 256) {
      const int r = i / CB_TK, cc = i % CB_TK;
      const int g = g0 + cc;
      sp[r][cc] = (b0 + r < nb && g < gend) ? psi[(size_t)(b0 + r) * npw + g] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < CB_TK; ++kk) {
      double2 x[PI], y[BJ];
#pragma unroll
      for (int i = 0; i < PI; ++i) x[i] = sb[tx + TX * i][kk];
#pragma unroll
      for (int j = 0; j < BJ; ++j) y[j] = sp[ty + TY * j][kk];
      // acc += conj(x) * y as four fused multiply-adds per complex product (written out so that
      // no separate multiply or add reaches the float64 pipe)
#pragma unroll
      for (int i = 0; i < PI; ++i)
#pragma unroll
        for (int j = 0; j < BJ; ++j) cmac_conj(acc[i][j], x[i], y[j]);
    }
    __syncthreads();
  }
  double2* out = part + (size_t)split * nb * nproj;
#pragma unroll
  for (int i = 0; i < PI; ++i)
#pragma unroll
    for (int j = 0; j < BJ; ++j) {
      const int p = p0 + tx + TX * i, b = b0 + ty + TY * j;
      if (p < nproj && b < nb) out[(size_t)b * nproj + p] = acc[i][j];
    }
}

__device__ __forceinline__ void calbec_tile(int npw, int nproj, int nb, int kchunk, const double2* __restrict__ beta,
                                            const double2* __restrict__ psi, double2* __restrict__ part, int tp,
                                            int tb, int split, double2* sm) {
  calbec_tile_t<CB_TP>(npw, nproj, nb, kchunk, beta, psi, part, tp, tb, split, sm);
}

// projectors per calbec tile for an item with nproj projectors
inline int calbec_tp(int nproj) { return nproj <= 8 ? 8 : (nproj <= 16 ? 16 : CB_TP); }


// w[b][p] = sum_{q in row p of D} D_pq sum_s part[s][b][q]
__device__ __forceinline__ void dscale_one(int i, int nproj, int nb, int nsplit, const double2* __restrict__ part,
                                           const int* __restrict__ rowptr, const int* __restrict__ col,
                                           const double2* __restrict__ val, double2* __restrict__ w) {
  if (i >= nproj * nb) return;
  const int b = i / nproj, p = i % nproj;
  double2 acc = make_double2(0.0, 0.0);
  for (int e = rowptr[p]; e < rowptr[p + 1]; ++e) {
    const int q = col[e];
    double2 s = make_double2(0.0, 0.0);
    for (int sp = 0; sp < nsplit; ++sp) {
      const double2 t = part[((size_t)sp * nb + b) * nproj + q];
      s.x += t.x;
      s.y += t.y;
    }
    const double2 d = val[e];
    acc.x += d.x * s.x - d.y * s.y;
    acc.y += d.x * s.y + d.y * s.x;
  }
  w[i] = acc;
}


constexpr int AV_TG = 64;   // G per CTA
constexpr int AV_TB = 32;   // bands per CTA
constexpr int AV_TP = 16;   // projectors per shared-memory tile

constexpr int AV_SMEM = AV_TP * AV_TG + AV_TB * (AV_TP + 1);   // double2 entries of shared memory

// hpsi[b][G] += sum_p w[b][p] beta[p][G]; sm: AV_SMEM entries of shared memory
__device__ __forceinline__ void addvus_tile(int npw, int nproj, int nb, const double2* __restrict__ w,
                                            const double2* __restrict__ beta, double2* __restrict__ hpsi, int tg,
                                            int tb, double2* sm) {
  auto sb = reinterpret_cast<double2 (*)[AV_TG]>(sm);                      // [AV_TP][AV_TG]
  auto sw = reinterpret_cast<double2 (*)[AV_TP + 1]>(sm + AV_TP * AV_TG);  // [AV_TB][AV_TP + 1]
  const int g0 = tg * AV_TG, b0 = tb * AV_TB;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // tx -> G, ty -> bands ty + 4 j
  double2 acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = make_double2(0.0, 0.0);
  for (int q0 = 0; q0 < nproj; q0 += AV_TP) {
    for (int i = threadIdx.x; i < AV_TP * AV_TG; i += 256) {
      const int r = i / AV_TG, cc = i % AV_TG;
      const int q = q0 + r, g = g0 + cc;
      sb[r][cc] = (q < nproj && g < npw) ? beta[(size_t)q * npw + g] : make_double2(0.0, 0.0);
    }
    for (int i = threadIdx.x; i < AV_TB * AV_TP; i += 256) {
      const int r = i / AV_TP, cc = i % AV_TP;
      const int b = b0 + r, q = q0 + cc;
      sw[r][cc] = (b < nb && q < nproj) ? w[(size_t)b * nproj + q] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < AV_TP; ++kk) {
      const double2 x = sb[kk][tx];
#pragma unroll
      for (int j = 0; j < 8; ++j) cmac(acc[j], sw[ty + 4 * j][kk], x);
    }
    __syncthreads();
  }
  const int g = g0 + tx;
  if (g < npw) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int b = b0 + ty + 4 * j;
      if (b < nb) {
        double2* o = hpsi + (size_t)b * npw + g;
        double2 v = *o;
        v.x += acc[j].x;
        v.y += acc[j].y;
        *o = v;
      }
    }
  }
}


// ---- many problems in one launch per kernel (hpsi_apply_batch) ----
// Each launch takes every item's geometry by value; CTA i finds its item from the running tile
// counts (at most kNlBatch items, a short scan) and then does exactly what the one-item kernel does.
constexpr int kNlBatch = 32;

struct NlItem {
  int npw, nproj, nb, kchunk, nsplit, tilesp, tilesb, gtiles;
  int tp;   // projectors per calbec tile (8, 16 or 32; 32 in the persistent launch)
  const double2* beta;
  const double2* psi;
  double2* hpsi;
  double2* part;
  double2* w;
  const int* rowptr;
  const int* col;
  const double2* dval;
};

struct NlBatch {
  int nitems;
  int off_cal[kNlBatch + 1];   // first calbec tile of each item (tilesp x tilesb x nsplit each)
  int off_ds[kNlBatch + 1];    // first D-scale block (256 outputs each)
  int off_add[kNlBatch + 1];   // first add_vuspsi tile (gtiles x tilesb)
  NlItem item[kNlBatch];
};

__device__ __forceinline__ int find_item(const int* off, int nitems, int blk) {
  int i = 0;
  while (i + 1 < nitems && off[i + 1] <= blk) ++i;
  return i;
}

