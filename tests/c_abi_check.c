/* Compiled (not run) by tests/test_abi.py: the public headers are plain C99
 * and declare what a C caller links against. */
#include <stddef.h>

#include "fs.h"
#include "fs_server.h"
#include "fs_stages.h"

int fs_c_abi_check(void) {
  fs_params p;
  fs_server_config c;
  size_t bytes = 0;
  fs_status (*create)(const fs_calib*, const fs_pose*, int, int, int, const fs_params*, void*,
                      fs_handle**) = fs_create;
  if (fs_default_params(&p) != FS_OK) return 1;
  if (fs_server_default_config(&c) != FS_OK) return 2;
  if (fs_state_bytes(64, 64, 2, &p, &bytes) != FS_OK) return 3;
  (void)create;
  (void)fs_solve;
  (void)fs_guard_check;
  return p.deriv == FS_DERIV_FORWARD && p.accel_gamma == 0.f && FS_STAGE_CLIP_WARP == 8 ? 0 : 4;
}
