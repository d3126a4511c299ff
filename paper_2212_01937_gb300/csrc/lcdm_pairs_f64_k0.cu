// Pair-kernel instantiations: precision f64, 0 tangent directions.
#include "lcdm_launch.cuh"
namespace lcdm {
LCDM_DEFINE_TABLE(table_f64_k0, 0, 0)
}
