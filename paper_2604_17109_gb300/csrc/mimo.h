// Host-side MIMO formulation and reconstruction (internal to the library).
#pragma once
#include <cstdint>

namespace pim {

// Spins per real symbol component (the correction depth) by default: 2 for 4-/16-QAM
// (T = [I, I], corrections {-2, 0, 2}), 3 for 64-QAM (T = [2I, I, I], corrections
// {-4, .., 4}); 0 for an unsupported constellation.
int mimo_spins_per_component(int qam);

// Correction depth of a request: depth 0 = the constellation's default, else 2 or 3 (any
// supported constellation); 0 when invalid.
int mimo_depth(int qam, int depth);

// DI-MIMO instance around the hard-sliced MMSE estimate (complex inputs interleaved re, im;
// H row-major nr x nt).  J_out: n x n, h_out: n, xm_ri: nt complex (interleaved), with
// n = depth * 2 nt (depth = mimo_depth(qam, depth)); library energy convention
// H(s) = -1/2 s^T J s - h^T s.
int mimo_formulate(int nt, int nr, int qam, const double* H_ri, const double* y_ri, double reg,
                   double* J_out, double* h_out, double* xm_ri, int depth = 0);

// x_ri (nt complex, interleaved) = slice(x_m + T s).
void mimo_reconstruct(int nt, int qam, const double* xm_ri, const int8_t* spins, double* x_ri,
                      int depth = 0);

}  // namespace pim
