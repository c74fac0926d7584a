// Temporary: tensor-core paths not yet linked in report "not supported".
#include "device.h"

namespace famlies {

int64_t emu_workspace_bytes(const Plan&) { return 0; }
cudaError_t launch_emu(const Plan&, const GemmArgs&, void*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace famlies
