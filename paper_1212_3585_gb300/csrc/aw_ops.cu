// aw_ops.cu -- selects the compiled hot-kernel instantiation for a configuration.
#include "aw_ops.h"

namespace aw {
HotOps ops_2_1_0();
HotOps ops_2_1_2();
HotOps ops_2_2_0();
HotOps ops_2_3_0();
HotOps ops_3_2_0();
HotOps ops_2_2_1();
HotOps ops_2_3_1();
HotOps ops_2_2_2();
HotOps ops_2_3_2();
HotOps ops_3_2_2();

bool get_ops(int D, int M, int PDE, HotOps* out) {
  int key = D * 100 + M * 10 + PDE;
  switch (key) {
    case 210: *out = ops_2_1_0(); return true;
    case 212: *out = ops_2_1_2(); return true;
    case 220: *out = ops_2_2_0(); return true;
    case 230: *out = ops_2_3_0(); return true;
    case 320: *out = ops_3_2_0(); return true;
    case 221: *out = ops_2_2_1(); return true;
    case 231: *out = ops_2_3_1(); return true;
    case 222: *out = ops_2_2_2(); return true;
    case 232: *out = ops_2_3_2(); return true;
    case 322: *out = ops_3_2_2(); return true;
  }
  return false;
}
}  // namespace aw
