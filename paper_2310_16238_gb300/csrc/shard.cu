// One rank's part of a fit sharded by stratum (arXiv 2310.16238, §2.1 eq. strat_l: the stratified
// partial likelihood is a sum over strata, and every risk-set sum a suffix sum within its
// stratum, §2.6-§2.7). The rows of one fit are cut into contiguous shards, one per rank; a rank
// holds a handle on its own rows and, per coordinate j, the ranks run in lock step:
//   head      the previous step's update at the shard's entries of its column (eta += x dbeta,
//             eq. parallel_xb; v = exp(eta), eq. parallel_d), then the shard's sums of v, x_j v and
//             x_j^2 v from its first row to its first stratum end (what the previous rank's last
//             stratum needs from this one);
//   partial   column j's (G1, G2) of eqs. (parallel_g)/(parallel_h) over the shard's tie groups,
//             its last stratum completed by the later ranks' sums (the carry), and, at the first
//             coordinate of a sweep, sum d log S0 and beta'dX over the shard -- the streaming
//             kernel in its shard mode;
//   step      from the ranks' summed partials: the convergence test at the first coordinate of a
//             sweep, then the Newton / L1 / trust-region step (§2.4) -- the same on every rank.
// The collectives between these calls (an all-gather of the head sums, an all-reduce of the
// partials) are the caller's.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ccd_common.cuh"
#include "cox.h"
#include "cox_internal.h"

namespace coxgb {

// Applies the pending update at column pend_j's entries, then sums v, x_j v, x_j^2 v over
// positions [0, cut_pos[0]] (one block, fixed summation order).
__global__ void __launch_bounds__(1024) shard_head_kernel(const DevFit *__restrict__ fit, int32_t j, double *out) {
  const DevFit &F = *fit;
  const DevData *D = F.d;
  FitCtl *ctl = F.ctl;
  const int tid = threadIdx.x;
  const int pj = ctl->pend_j;
  const double db = ctl->pend_db;
  if (pj >= 0) {
    for (int64_t q = D->col_ptr[pj] + tid; q < D->col_ptr[pj + 1]; q += blockDim.x) {
      const uint32_t e = D->idx[q];
      const int64_t pos = e & kPosMask;
      const double x = D->val ? D->val[q] : 1.0;
      const double et = __dadd_rn(F.eta[pos], __dmul_rn(x, db));
      F.eta[pos] = et;
      static_cast<double *>(F.v)[pos] = make_v<PF64>(et, F.shift, (e & kExitBit) != 0, &ctl->error);
    }
  }
  __syncthreads();
  __threadfence_block();
  const int64_t last = D->K > 0 ? D->cut_pos[0] : -1;   // the first stratum end (or the data's end)
  double acc[3] = {0.0, 0.0, 0.0};
  const double *v = static_cast<const double *>(F.v);
  for (int64_t pos = tid; pos <= last; pos += blockDim.x) acc[0] += v[pos];
  if (j >= 0)
    for (int64_t q = D->col_ptr[j] + tid; q < D->col_ptr[j + 1]; q += blockDim.x) {
      const int64_t pos = D->idx[q] & kPosMask;
      if (pos > last) break;   // a column's entries are ascending
      const double x = D->val ? D->val[q] : 1.0;
      acc[1] += x * v[pos];
      acc[2] += x * x * v[pos];
    }
  __shared__ double s[3][32];
  for (int i = 0; i < 3; ++i)
    for (int off = 16; off > 0; off >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], off);
  if ((tid & 31) == 0)
    for (int i = 0; i < 3; ++i) s[i][tid >> 5] = acc[i];
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) {
      double r = 0.0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) r += s[i][w];
      out[i] = r;
    }
    out[3] = 0.0;
    ctl->pend_j = -1;   // applied
  }
}

// The convergence test (when due) and the coordinate step of column j from the ranks' summed
// partials tot = (G1, G2, sum d log S0, beta'dX); out = (state, loglik).
__global__ void __launch_bounds__(256) shard_step_kernel(const DevFit *__restrict__ fit, const double *__restrict__ dxg,
                                                         int32_t j, double g1s, double g2s, double lls, double bdx,
                                                         int32_t need_ll, int32_t sweep, int32_t max_sweeps,
                                                         double *out) {
  const DevFit &F = *fit;
  const DevData *D = F.d;
  FitCtl *ctl = F.ctl;
  const int tid = threadIdx.x;
  double pen = 0.0;
  if (need_ll) {
    for (int jj = tid; jj < D->p; jj += blockDim.x) {
      const double b = F.beta[jj];
      const bool pz = F.penalize ? F.penalize[jj] != 0 : true;
      if (pz && F.penalty == COX_PEN_L1) pen += F.lambda * fabs(b);
      if (pz && F.penalty == COX_PEN_L2) pen += b * b / (2.0 * F.l2_var);
    }
    __shared__ double s[32];
    for (int off = 16; off > 0; off >>= 1) pen += __shfl_down_sync(0xffffffffu, pen, off);
    if ((tid & 31) == 0) s[tid >> 5] = pen;
    __syncthreads();
    if (tid == 0) {
      pen = 0.0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) pen += s[w];
    }
  }
  if (tid != 0) return;
  int state = kRunning;
  double ll = 0.0;
  if (need_ll) {
    ll = bdx - lls;
    const double obj = -ll + pen;
    ctl->loglik = ll;
    ctl->obj = obj;
    if (sweep > 0 && fabs(obj - ctl->obj_prev) <= F.tol * fabs(obj)) state = kConverged;
    else if (sweep >= max_sweeps) state = kMaxed;
    else ctl->obj_prev = obj;
  }
  if (ctl->error) state = kError;
  if (state == kRunning) {
    const int pz = F.penalize ? F.penalize[j] != 0 : 1;
    double tr = F.trust[j];
    const double s = ccd_step_rule(-dxg[j] + g1s, g2s, F.beta[j], &tr, F.penalty, F.lambda, F.l2_var, pz);
    F.trust[j] = tr;
    if (s != 0.0) {
      F.beta[j] = F.beta[j] + s;
      ctl->pend_j = j;
      ctl->pend_db = s;
    } else {
      ctl->pend_j = -1;
    }
    ctl->coord_updates += 1;
  }
  ctl->state = state;
  ctl->sweep = sweep;
  out[0] = double(state);
  out[1] = ll;
}

// Removes the data's last stratum end from the last tile's list (the stratum continues on the
// next rank), so that the streaming kernel's last tile takes lc->ext as its carry.
__global__ void shard_open_end_kernel(DevData *d, int32_t *tile_k) {
  if (threadIdx.x == 0 && d->K > 0) tile_k[d->T] = d->K - 1;
}

int launch_shard_head(const DevFit *fit, int32_t j, double *out, void *stream) {
  count_launches(1);
  shard_head_kernel<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(fit, j, out);
  return cudaPeekAtLastError() == cudaSuccess ? COX_OK : COX_E_CUDA;
}

int launch_shard_step(const DevFit *fit, const double *dxg, int32_t j, const double *tot, int32_t need_ll, int32_t sweep,
                      int32_t max_sweeps, double *out, void *stream) {
  count_launches(1);
  shard_step_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(fit, dxg, j, tot[0], tot[1], tot[2], tot[3],
                                                                       need_ll, sweep, max_sweeps, out);
  return cudaPeekAtLastError() == cudaSuccess ? COX_OK : COX_E_CUDA;
}

int launch_shard_open_end(DevData *d, int32_t *tile_k, void *stream) {
  count_launches(1);
  shard_open_end_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(d, tile_k);
  return cudaPeekAtLastError() == cudaSuccess ? COX_OK : COX_E_CUDA;
}

}  // namespace coxgb
