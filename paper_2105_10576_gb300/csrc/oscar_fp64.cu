// FP64 path: every field, stencil and multigrid level in double.
#include "oscar_solver.cuh"
namespace oscar {
template struct Solver<double>;
}
