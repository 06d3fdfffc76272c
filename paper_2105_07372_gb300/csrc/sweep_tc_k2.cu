// Split-sweep transform kernel (tcgen05) instances for K+1 up to 48 (rows in steps of 4).
#include "sweep_tc_impl.cuh"

namespace mra {
SplitTransFn sweep_tc_trans(int KP) {
  switch (KP) {
    case 4: return k_tc_trans<4>;
    case 8: return k_tc_trans<8>;
    case 12: return k_tc_trans<12>;
    case 16: return k_tc_trans<16>;
    case 20: return k_tc_trans<20>;
    case 24: return k_tc_trans<24>;
    case 28: return k_tc_trans<28>;
    case 32: return k_tc_trans<32>;
    case 36: return k_tc_trans<36>;
    case 40: return k_tc_trans<40>;
    case 44: return k_tc_trans<44>;
    case 48: return k_tc_trans<48>;
    default: return nullptr;
  }
}
}  // namespace mra
