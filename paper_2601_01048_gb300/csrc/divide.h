// Device opcode of a checked division (DIV / REM of the program format),
// numbered after the shared layout's opcodes: the loader emits it and the
// bytecode interpreter executes it.  Programs compiled at load time carry
// their divisions as emitted code.
#pragma once

#include "layout.h"

namespace cufz {

// DevOp fields: d = quotient or remainder register, a = dividend, b =
// divisor, imm = division site, x = 1 for REM | 2 when the result is live.
constexpr uint8_t D_DIVREM = D_NUM_OPCODES;

}  // namespace cufz
