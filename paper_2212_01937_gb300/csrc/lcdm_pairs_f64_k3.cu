// Pair-kernel instantiations: precision f64, 3 tangent directions.
#include "lcdm_launch.cuh"
namespace lcdm {
LCDM_DEFINE_TABLE(table_f64_k3, 0, 3)
}
