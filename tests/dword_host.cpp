// Host build of the double-word arithmetic used by the bus kernel (the same
// header the CUDA library compiles), for the CPU tests of its error bounds
// and the GPU test that compares the device's bits with these.
#include "dword.cuh"

extern "C" void dw_host_ops(int op, int n, const double *x, const double *y, const double *z, double *out) {
  for (int i = 0; i < n; ++i) ucac::dw_probe_op(op, x[i], y[i], z[i], out + 4 * (long)i);
}
