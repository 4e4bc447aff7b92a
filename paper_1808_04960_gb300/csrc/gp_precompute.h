// Host-side GP weight precompute in double-double arithmetic (Section 4, step 1).
#pragma once
#include <cstddef>

namespace gpweno {

constexpr int kMaxR = 3;
constexpr int kMaxS = kMaxR + 1;           // points per sub-stencil
constexpr int kMaxBig = 2 * kMaxR + 1;     // points of the full stencil

struct GpTables {
    int R;
    // left state of face i+1/2 (x* = +1/2 from the stencil of cell i)
    double wl[kMaxS * kMaxS];   // [m][j]
    double gl[kMaxS];
    double wbig_l[kMaxBig];
    // right state of face i+1/2 (x* = -1/2 from the stencil of cell i+1)
    double wr[kMaxS * kMaxS];
    double gr[kMaxS];
    double wbig_r[kMaxBig];
    // smoothness factors P[h][j] = v_h[j] / sqrt(lambda_h) of K_m(sigma), lambda ascending
    double P[kMaxS * kMaxS];
    double lambda[kMaxS];
    // The same factors in half form, largest eigenvalue first: K_m(sigma) is
    // symmetric Toeplitz, hence persymmetric, and the SE kernel is totally
    // positive, so in descending order of lambda the eigenvectors alternate
    // symmetric (k even: v_j = v_{S-1-j}) and skew (k odd: v_j = -v_{S-1-j}).
    // Ph[k*S + j], j < (S+1)/2, holds the first half of P for the k-th largest
    // eigenvalue; the precompute verifies the alternation.
    double Ph[kMaxS * kMaxS];
    double Psum[kMaxS];          // sum_j P_kj of each full row, same order as Ph (0 for skew rows)
    double sl1[kMaxS];           // sum_j wl[m][j] - 1, from the double-double weights
    double sr1[kMaxS];           // sum_j wr[m][j] - 1
    // the same scaled by the linear weights, for the weighted sum of Eq. weight_sum:
    // gwl[m][j] = gl[m] wl[m][j], gsl1[m] = gl[m] sl1[m] (and right)
    double gwl[kMaxS * kMaxS], gwr[kMaxS * kMaxS], gsl1[kMaxS], gsr1[kMaxS];
    double ls_residual;          // ||M gamma - w||_2 of the left-state system
    double cond_estimate;        // rough condition estimate of K(l)
};

// Returns 0 on success; otherwise writes a message to err and returns
// 1 (bad argument) or 2 (ill-conditioned beyond double-double).
// poly = 1: candidate and full-stencil weights are polynomial instead of GP
// weights (the WENO-GP hybrid); the linear weights, K_m(sigma) and P are
// computed as usual.  recon = 1: the weights predict a point value from cell
// averages (reconstruction, for the FD-Flux form) instead of from point values.
int gp_precompute(int R, double ell_over_dx, double sigma_over_dx, GpTables *out, char *err, std::size_t errlen,
                  int poly = 0, int recon = 0);

// GP-AO tables (Appendix A): R = 2 serves AO(2,3), R = 3 the recursive
// AO(3,2,3).  GP weights of the full stencil S_R (hi), of S_{R-1} (lo, R = 3
// only) and of the three 3-point stencils of Eq. cweno_stencil (w3[m][j]),
// for the left (x* = +1/2) and right (x* = -1/2) states, each with its sum
// minus one; the smoothness factors of K_N(sigma) for N = 2R+1, 2R-1 and 3
// (full and half form as in GpTables, rows of length N) and log det K_N.
struct AoTables {
    int R;
    double w_hi_l[kMaxBig], w_hi_r[kMaxBig], s_hi_l, s_hi_r;
    double w_lo_l[kMaxBig], w_lo_r[kMaxBig], s_lo_l, s_lo_r;
    double w3_l[9], w3_r[9], s3_l[3], s3_r[3];
    double P_hi[kMaxBig * kMaxBig], Ph_hi[kMaxBig * kMaxBig], Psum_hi[kMaxBig], logdet_hi;
    double P_lo[kMaxBig * kMaxBig], Ph_lo[kMaxBig * kMaxBig], Psum_lo[kMaxBig], logdet_lo;
    double P_3[9], Ph_3[9], Psum_3[3], logdet_3;
};

int ao_precompute(int R, double ell_over_dx, double sigma_over_dx, AoTables *out, char *err, std::size_t errlen);

}  // namespace gpweno
