// Host tables of the reverse-time march (built from the plan's tables when the adjoint runs).
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace wave1d {

// The receivers' local weights (LocalCSR rloc: one row per receiver, m >= 0) regrouped by source:
// for source l, entries [src_ptr[l], src_ptr[l + 1]) in increasing receiver order, each with the
// receiver, its m range (m_lo | count << 16, as in LocalCSR) and the offset of its weights in
// rloc.w.  The receivers' transposed readout then has one writer per source.
struct ReceiverColumns {
    std::vector<int64_t> src_ptr;
    std::vector<int32_t> rcv;
    std::vector<int32_t> mrange;
    std::vector<int64_t> woff;
};
void receiver_columns(const LocalCSR& rloc, int64_t M, ReceiverColumns& out);

}  // namespace wave1d
