// flow_tables.hpp -- the FLOW form's host-built tables (built in inspect.cpp,
// uploaded by the runtime at a sim's first FLOW step, read by flow.cuh).
#pragma once
#include <cstdint>
#include <vector>

#include "lower.hpp"

namespace rteaal {

// The kernel's stamped words are indexed by row in layout order: class-3 rows
// first, then 2, 1, 0, each class in reference order.  op: 8 words per lowered
// op -- rows of operands a, b, c (FLOW_CHECK on a row an op writes in the
// cycle, whose stamp the item waits for; 0 for an absent operand and for ops
// with more than three operands), the output's row, ctl, the output's
// reference, the side-array offset and the operand count (extended ops only).
// ext: the rows of the extended ops' operands, flagged the same way.  pool:
// {reference, row} of every input, register and constant, in that order.
constexpr uint32_t FLOW_CHECK = 1u << 31;
void flow_tables(const Lowered& L, std::vector<uint32_t>& op, std::vector<uint32_t>& ext,
                 std::vector<uint32_t>& pool);

}  // namespace rteaal
