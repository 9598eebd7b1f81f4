/* Test hooks of the bounds-checked build of libfbp (libfbp_checked.so, compiled with
 * FBP_BOUNDS_CHECK); the ordinary library does not export them.  No counterpart in the paper.
 *
 * In the checked build every kernel of the reconstruction, its adjoints and SIRT checks each
 * global index it forms against its buffer (and the shared-memory range of each Hough
 * round); every build checks that each geometry-table row it uses names angle rows inside
 * the sinogram.  A failed check skips the access and records FBP_ERR_INTERNAL in the plan's
 * status word (fbp_last_device_error).  The corrector's kernels check their global indices
 * and bulk-copy ranges the same way and record FBP_ERR_INTERNAL in the corrector's status
 * word (fbp_cnn_last_error); a skipped bulk copy leaves its stage unfilled, so the bounded
 * wait for it expires and the CTA stops. */
#ifndef FBP_CHECK_H
#define FBP_CHECK_H

#include "fbp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Overwrite the first angle row k0 of geometry-table row (quarter q, slope row i) of the
 * plan (synchronises the device first).  With k0 outside [0, K-1] (or not K-1 on the row
 * that wraps past the last angle) the kernels reject that row: they validate it before any
 * access, resample it as zeros and set the status word.  For tests of the status word; the
 * plan's results are meaningless afterwards.
 * Errors: FBP_ERR_INVALID_ARG (NULL plan, q outside 0..3, i outside 0..N-1), FBP_ERR_CUDA. */
fbp_status fbp_check_set_row_angle(fbp_plan_t plan, int q, int i, int k0);

/* Make the corrector's last layer (fbp_cnn_forward) check its image loads and stores as if
 * the call had `images` images (0: the call's own count again; synchronises the device
 * first).  With fewer images than the call has, the pixels of the later images fail the
 * check: their loads read 0, their outputs are not written, and fbp_cnn_last_error returns
 * FBP_ERR_INTERNAL.  Process-wide setting, for tests of the corrector's status word.
 * Errors: FBP_ERR_INVALID_ARG (images < 0), FBP_ERR_CUDA. */
fbp_status fbp_check_cnn_image_limit(int images);

#ifdef __cplusplus
}
#endif

#endif /* FBP_CHECK_H */
