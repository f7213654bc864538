// Launch wrappers of the flattened kernels over a ragged batch (ragged.cuh):
// each takes one entry per problem (its grid with one right-hand side, its
// operator, vectors and buffers) and launches every kernel once over all of
// them, in groups of at most RMAXP problems.
#pragma once
#include <vector>

#include "internal.h"

namespace hmg {

// One problem's smoothing or transfer at one level.
template <class T> struct RagLevel {
  Grid g;            // the problem's grid at this level (one right-hand side)
  OpView<T> op;      // its operator at this level
  cx<T>* x;          // iterate
  const cx<T>* b;    // right-hand side
  GmresBufs gb;      // GMRES(3) vectors, scalars, reduction partials and ticket
  const int* active; // the problem's convergence mask
};

// nu GMRES(3) smoothing steps of the fine level (row marches), of a
// Kronecker-form level (column marches); the update and the closing
// Arnoldi pass shared by both.
template <class T> void gmres_smooth_march_rag(const std::vector<RagLevel<T>>& v, int nu, cudaStream_t s,
                                               cudaStream_t side, cudaEvent_t fork, cudaEvent_t join);
template <class T> void gmres_smooth_kron_rag(const std::vector<RagLevel<T>>& v, int nu, cudaStream_t s);
template <class T> void launch_gmres_update_rag(const std::vector<RagLevel<T>>& v, cudaStream_t s);
// g_arn_b<J> on every problem; un_next: store u_{J+1} (into u[J+1]); ws as g_arn_b
template <class T, int J> void launch_arn_b_rag(const std::vector<RagLevel<T>>& v, bool un_next, int ws,
                                                cudaStream_t s);

// One problem's inter-grid transfer between level l (fine) and l + 1.
template <class T> struct RagXfer {
  Grid gf, gc;
  OpView<T> op;        // the fine level's operator
  const cx<T>* x;      // fine iterate
  const cx<T>* b;      // fine right-hand side
  cx<T>* rc;           // coarse right-hand side (restriction) or coarse correction (prolongation input)
  cx<T>* xf;           // fine iterate to correct (prolongation)
  const int* active;
};
template <class T> void launch_resid_restrict_rag(const std::vector<RagXfer<T>>& v, const Xfer& xw, cudaStream_t s);
template <class T> void launch_prolong_add_rag(const std::vector<RagXfer<T>>& v, const Xfer& xw, cudaStream_t s);

// Zero a vector of each problem (its grid with one right-hand side).
struct RagVec {
  Grid g;
  void* v;
  const int* active;
};
template <class T> void launch_zero_rag(const std::vector<RagVec>& v, cudaStream_t s);

// The refinement loop of the mixed path and the FP64 stopping test.
struct RagOuter {
  Grid g;
  Op0<double> op;
  double2* x;          // FP64 outer iterate
  const double2* b;    // FP64 right-hand side
  float2* e;           // complex64 correction (mixed) / residual output (mixed)
  float2* r32;
  Ctl c;
};
void launch_update_mixed_rag(const std::vector<RagOuter>& v, cudaStream_t s);
void launch_resid_cast_stop_rag(const std::vector<RagOuter>& v, int count, cudaStream_t s);
void launch_resnorm_stop_rag(const std::vector<RagOuter>& v, int count, cudaStream_t s);

// One visit of each problem's coarse sub-cycle (one CTA per problem).
template <class T> struct RagCoarse {
  const CLevel<T>* levels;
  const CStep* steps;
  int nsteps;
  const double2* inv;
  int N;
  const int* active;
};
template <class T> void launch_coarse_cycle_rag(const std::vector<RagCoarse<T>>& v, cudaStream_t s);

// out[p] = the active count of problem p ([0] of its count pair), out[np + p]
// = its barrier-error flag ([1]).
void launch_gather_counts(const std::vector<const int*>& counts, int* out, cudaStream_t s);

}  // namespace hmg
