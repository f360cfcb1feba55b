// Device accumulation of the Gaussian sketch behind the interpolative decomposition of
// the one-patch far field (Kaye & Greengard, Section 7.1): Y (ks x nf, column-major)
// += Omega[:, r0:r1] A[r0:r1, :] with A_tl = G(|x_t - x_l|), the on-surface Green's
// function between training target t and fine-grid point l. Host-only interface (no CUDA
// types), used by the precompute when a CUDA device is available.
#pragma once

namespace ncs {

struct DeviceSketch;

// Uploads Omega (ks x nt, row-major), the training targets xt (nt x 3) and the fine-grid
// points xf (nf x 3) and zeroes Y on the current device. mode: 0 exterior, 1 interior.
// Returns null if no device is usable or an allocation fails.
DeviceSketch* sketch_create(int ks, int nt, int nf, int mode, const double* Om, const double* xt,
                            const double* xf);
// Y += Omega[:, r0:r1] A[r0:r1, :] (asynchronous). Returns false on a CUDA error.
bool sketch_add_rows(DeviceSketch* s, int r0, int r1);
// Copies the running Y (ks * nf doubles, column-major) to host memory.
bool sketch_read(DeviceSketch* s, double* Y);
void sketch_destroy(DeviceSketch* s);

}  // namespace ncs
