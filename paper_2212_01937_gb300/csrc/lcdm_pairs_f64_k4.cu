// Pair-kernel instantiations: precision f64, 4 tangent directions.
#include "lcdm_launch.cuh"
namespace lcdm {
LCDM_DEFINE_TABLE(table_f64_k4, 0, 4)
}
