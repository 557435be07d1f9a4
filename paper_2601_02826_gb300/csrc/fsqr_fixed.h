// Launchers of the setup passes on exact integer products (k_setup.cu,
// k_iter.cu): the power method's X~_g v and X~_g^T u for eta_g (Section 4)
// and the X~^T v of lambda_max, with the vector in 52-bit fixed point.
#pragma once

#include "fsqr_internal.h"

namespace fsqr {

// Rounds x (times mult, when given) per segment to q = hi 2^26 + lo,
// 0 <= lo < 2^26, with unit[s] = 2^(e-52), 2^e > max |x mult| over the
// segment; entries below `first` get q = 0. cst[s] = sum of cmul_k x_k over
// the rounded entries (cmul, cst NULL: none). Segments come from bounds
// (2 per segment) or, with bounds NULL, are seglen entries each.
cudaError_t launch_fix_seg(const double *x, const double *mult, const double *cmul, const int64_t *bounds,
                           int64_t seglen, int nseg, int64_t first, int2 *q, double *unit, double *cst,
                           cudaStream_t s);
// launch_xv_blocks for int8/2-bit storage from launch_fix_seg's output over
// the splits (mult = a, cmul = b, first = c + 1).
cudaError_t launch_xv_blocks_int(const Dsg &X, const double *v, const int64_t *splits, const int *split_of_block,
                                 int G, int nsplit, const int2 *q, const double *unit, const double *cst, double *u,
                                 int64_t npad, double *part, cudaStream_t s);
// s_out[j] = x~_j^T u_g(j) from u (FP64, npad per block) and its fixed point
// per block; G = 1 with block_ptr NULL gives one vector for every column.
cudaError_t launch_xtv_int(const Dsg &X, const int64_t *block_ptr, int G, const double *u, const int2 *q,
                           const double *unit, const double *usum, int64_t npad, double *s_out, cudaStream_t s);

}  // namespace fsqr
