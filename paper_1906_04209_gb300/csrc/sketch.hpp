// The interpolative decompositions of the one-patch far field (Kaye & Greengard,
// Section 7.1) on the device: the Gaussian sketch Y (ks x nf, column-major) += Omega[:, r0:r1]
// A[r0:r1, :] with A_tl = G(|x_t - x_l|), the on-surface Green's function between training
// target t and fine-grid point l; the column-pivoted QR of its leading rows; the outgoing
// operator T. Host-only interface (no CUDA types), used by the precompute when a CUDA
// device is available.
#pragma once

#include <vector>

namespace ncs {

struct DeviceSketch;

// Uploads Omega (ks x nt, row-major), the training targets xt (nt x 3) and the fine-grid
// points xf (nf x 3) and zeroes Y on the current device. mode: 0 exterior, 1 interior.
// ff: form the sketch in float-float on the FP32 pipes (Omega's values must then be FP32
// numbers; kernel entries accurate to ~1e-14 relative, for ID tolerances from 1e-12 up),
// else in FP64. Returns null if no device is usable or an allocation fails.
DeviceSketch* sketch_create(int ks, int nt, int nf, int mode, const double* Om, const double* xt,
                            const double* xf, bool ff);
// Y += Omega[:, r0:r1] A[r0:r1, :] (asynchronous). Returns false on a CUDA error.
bool sketch_add_rows(DeviceSketch* s, int r0, int r1);
// Copies the running Y (ks * nf doubles, column-major) to host memory.
bool sketch_read(DeviceSketch* s, double* Y);
void sketch_destroy(DeviceSketch* s);

// Column-pivoted Householder QR, on the device, of the first kse rows of the running
// sketch (a copy; the sketch keeps accumulating), stopped at |R_kk| < tol |R_00| (pivot
// ties pick the lowest column). Returns the rank p, or -1 on a CUDA error; piv receives
// the column order (nf entries).
int sketch_cpqr(DeviceSketch* s, int kse, double tol, std::vector<int>& piv);
// Uploads the W B rows of the fine-grid points (nf x K, row-major) used by sketch_assemble.
bool sketch_set_wb(DeviceSketch* s, int K, const double* WB);
// After sketch_cpqr of rank p: T (p x K, row-major) = W B[piv[:p]] + X W B[piv[p:]] with
// X = R11^-1 R12 from that factorisation (eq. Tmap). Returns false on a CUDA error.
bool sketch_assemble(DeviceSketch* s, int p, std::vector<double>& T);

}  // namespace ncs
