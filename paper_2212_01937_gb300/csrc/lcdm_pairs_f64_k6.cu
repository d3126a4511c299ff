// Pair-kernel instantiations: precision f64, 6 tangent directions.
#include "lcdm_launch.cuh"
namespace lcdm {
LCDM_DEFINE_TABLE(table_f64_k6, 0, 6)
}
