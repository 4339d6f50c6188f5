// Mixed path: FP32 fields, stencils and V-cycles; the CG vectors, dot
// products, norms, phase-volume sums and relaxation accumulators stay FP64, so
// the pressure solve is an FP64 iteration preconditioned in FP32.
#include "oscar_solver.cuh"
namespace oscar {
template struct Solver<float>;
}
