// Upload preparation: the interface between the host runtime (api.cu) and its device
// launches (upload.cu). Kept apart from the pair kernels' shared header.
#ifndef HK_UPLOAD_H
#define HK_UPLOAD_H

#include "hk_internal.h"

namespace hk {

// Two launches form, from the float64 coordinates of n events (read from sx, sy, st; written to
// the set's x64, y64, t64 and padded there to npad): the float32 copies, the tie indices
// lo32/lo64, the window tables (first[nb] then last[nb], nullptr for none, buckets of `width`
// from t0 over the float32 or float64 times) and the input checks (flags |= 1: a value out of
// range or not finite; |= 2: times decrease). flags must be zero before the launch.
struct UploadPrep {
  const double *sx, *sy, *st;  // the caller's coordinates: host memory the device can read, or x64..
  double *x64, *y64, *t64;
  float *x32, *y32, *t32;
  int *lo32, *lo64;
  int *w32, *w64;
  double t0_32, width_32, t0_64, width_64;
  unsigned *flags;
  int64_t n, npad;
  int sms;  // multiprocessors of the device (sizes the grid)
};
cudaError_t launch_upload_prep(const UploadPrep &u, cudaStream_t s);

}  // namespace hk

#endif  // HK_UPLOAD_H
