// Host tables of a batched plan: many independent periodic instances (own springs, stiffnesses,
// incident pulse and receivers) sharing dt, N_t, tol and p, marched together.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "../../include/wave1d.h"

namespace wave1d {

// The instances' own plans (built by build_host_plan / build_receivers) joined into one table set
// in instance-major order: spring j of instance b is global spring moff[b] + j (both in the
// instance's internal, position-sorted order and in the caller's order), receiver r of instance b
// is roff[b] + r.  The joined plan `g` holds what the local sum, the block solve and the receivers
// read (items, m = 0 receiver terms, blocks, solve groups, stiffnesses, permutation) with every
// index moved by its instance's offsets; its history tables (FIR, rotation, mode factors,
// twiddles) are instance 0's, which all instances share.  inst_of: the instance of each global
// spring.  Returns 0, or WAVE1D_EINVAL (err set) if the instances' derived sizes differ.
struct BatchTables {
    HostPlan g;
    std::vector<int64_t> moff, roff;
    std::vector<int32_t> inst_of;
};
int join_instances(const std::vector<HostPlan>& inst, BatchTables& out, std::string& err);

// The two sizes that choose an instance's form in a batched plan with opts.local_weights = 2, from
// its positions alone (periodic box, positions wrapped into [-pi, pi)):
//   largest_block: members of the largest block of springs closer than dt (eq. linearSystem's
//     nearby graph; in 1D the runs of sorted neighbours less than dt apart, across the seam too);
//   pairs: ordered (target, source) pairs of distinct springs closer than delta (the local sum's).
// An instance is planned without pair lists when largest_block > max_block or pairs > kBatchPairs.
struct InstanceShape {
    int64_t largest_block = 0, pairs = 0;
};
InstanceShape instance_shape(const double* x, int64_t M, double dt, double delta);
constexpr int64_t kBatchPairs = (int64_t)1 << 19;

// The instances of a batched plan (arguments as wave1d_batch_plan) split by form, and the joined
// ones' own tables built in instance order against one weight budget: form[b] = 0 for a joined
// instance, 1 for one planned without pair lists (opts.local_weights 0: all joined, 1: none,
// 2: instance_shape's rule, and an instance whose stored weights would pass what is left of
// opts.max_local_bytes also goes without pair lists).  joined: the joined instances' indices, inst
// their tables (build_host_plan, build_receivers).  Returns 0, or the status of the first joined
// instance that cannot be built (err names it).  opts must hold defaults for max_block and
// max_local_bytes (> 0).
int batch_instances(int n_inst, const int64_t* offsets, const double* x, const double* beta,
                    const int64_t* r_offsets, const double* xr, double dt, int64_t Nt, double tol,
                    const wave1d_opts& o, std::vector<int>& form, std::vector<int>& joined,
                    std::vector<HostPlan>& inst, std::string& err);

}  // namespace wave1d
