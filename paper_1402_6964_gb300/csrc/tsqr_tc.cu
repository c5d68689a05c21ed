// tsqr_tc.cu -- tensor-core (tcgen05, TF32x3) form of the leaf pass.
#include "internal.h"

namespace mrnmf {

bool tc_supported(int n)
{
    (void)n;
    return false;
}

}  // namespace mrnmf
