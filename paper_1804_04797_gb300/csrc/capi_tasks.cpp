// C ABI of the few-amplitude task: amplitudes by the cut decomposition (K6) and by the
// inner product of a forward and a backward state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/sv.h"
#include "capi_util.h"
#include "kernels.h"
#include "plan.h"
#include "state.h"

using namespace svc;

namespace {

struct Holder {  // destroys a handle on scope exit
  sv_state *s = nullptr;
  ~Holder() { if (s) sv_destroy(s); }
};

sv_status generate(const sv_lattice *lat, std::vector<sv_gate> *g) {
  size_t n = 0;
  sv_status st = sv_generate_circuit(lat, nullptr, 0, &n);
  if (st != SV_OK) return st;
  g->resize(n);
  return sv_generate_circuit(lat, g->data(), n, &n);
}

int lattice_qubits(const sv_lattice *lat) {
  const int sites = lat->rows * lat->cols;
  int n = 0;
  for (int i = 0; i < sites; ++i) n += !((lat->removed_mask >> i) & 1ull);
  return n;
}


// How a cut is decomposed: the half gate lists (branch bits appended as qubits) and, per
// crossing CZ, its role.
struct CutPlan {
  int n = 0, na = 0, nb = 0;
  int local[64];
  bool in_a[64];
  int t = 0;          // crossing CZs
  int absorbed = 0;   // expanded into an output sign instead
  int tf = 0;         // branch bits in both halves (summed over)
  int ta = 0, tb = 0; // branch bits of half A / half B (tf + implicit ones of the other side)
  std::vector<svp::Gate> ga, gb;
  std::vector<svp::Gate> part_c;  // layers after the cut depth, on the full state (qubits as in the lattice)
  // output signs (-1)^{x_a x_b} of absorbed CZs; bits of x fixing implicit branch bits
  std::vector<std::pair<int, int>> signs;
  std::vector<std::pair<int, int>> fix_a;  // (branch bit index in A above na + tf, qubit of x)
  std::vector<std::pair<int, int>> fix_b;
};

// allow_implicit: may a crossing CZ be decomposed implicitly (an amplitude sum can fix
// the branch index by the output bit; a full-state product cannot)
sv_status plan_cut(const sv_lattice *lat, const sv_cut *cut, CutPlan *C, bool allow_implicit = true) {
  std::vector<sv_gate> g;
  sv_status st = generate(lat, &g);
  if (st != SV_OK) return st;
  const int n = C->n = lattice_qubits(lat);
  int &na = C->na, &nb = C->nb;
  na = nb = 0;
  for (int q = 0; q < n; ++q) {
    C->in_a[q] = (cut->half_a_mask >> q) & 1ull;
    C->local[q] = C->in_a[q] ? na++ : nb++;
  }
  if (na < 1 || nb < 1) return fail(SV_ERR_ARG, "sv_branch_amplitudes: both halves need qubits");
  if (cut->depth < 0) return fail(SV_ERR_ARG, "sv_cut: depth must be >= 0");
  const uint32_t depth = cut->depth > 0 ? (uint32_t)cut->depth : 0xffffffffu;
  // last non-diagonal gate of each qubit (H, square roots)
  std::vector<long> last_nd(n, -1);
  for (size_t i = 0; i < g.size(); ++i) {
    const int k = g[i].kind;
    if (k == SV_H || k == SV_SX || k == SV_SY || k == SV_SXDG || k == SV_SYDG) last_nd[g[i].q0] = (long)i;
  }
  // roles: 0 = full (projector on A, Z on B), 1 = absorbed sign, 2 = implicit on A (A's
  // qubit stays a basis state: no branch bit in A), 3 = implicit on B
  std::vector<int> role;
  for (size_t i = 0; i < g.size(); ++i) {
    const sv_gate &x = g[i];
    if (x.kind != SV_CZ || C->in_a[x.q0] == C->in_a[x.q1] || x.layer > depth) continue;
    const int qa = C->in_a[x.q0] ? x.q0 : x.q1, qb = C->in_a[x.q0] ? x.q1 : x.q0;
    const bool qa_quiet = last_nd[qa] < (long)i, qb_quiet = last_nd[qb] < (long)i;
    int r = 0;
    if (!cut->full_decomposition) r = (qa_quiet && qb_quiet) ? 1 : !allow_implicit ? 0 : qa_quiet ? 2 : qb_quiet ? 3 : 0;
    role.push_back(r);
  }
  C->t = (int)role.size();
  int n_full = 0, n_impl_a = 0, n_impl_b = 0;
  for (int r : role) {
    if (r == 0) ++n_full;
    if (r == 1) ++C->absorbed;
    if (r == 2) ++n_impl_a;
    if (r == 3) ++n_impl_b;
  }
  C->tf = n_full;
  C->ta = n_full + n_impl_b;  // A carries the Z^l side of CZs implicit on B
  C->tb = n_full + n_impl_a;
  if (na + C->ta > 34 || nb + C->tb > 34)
    return fail(SV_ERR_ARG, "sv_branch_amplitudes: half qubits + branch bits must be <= 34");
  // Half gate lists: every qubit, branch bits included, starts with H, so each branch
  // slice holds its half's state times 2^{-t_half/2}.  Branch bit numbering: the full
  // ones first (shared order), then the implicit ones of the other side.
  for (int q = 0; q < na + C->ta; ++q) C->ga.push_back(svp::Gate{svp::K_H, (uint8_t)q, 0});
  for (int q = 0; q < nb + C->tb; ++q) C->gb.push_back(svp::Gate{svp::K_H, (uint8_t)q, 0});
  int jf = 0, ja = 0, jb = 0, c = 0;
  for (const sv_gate &x : g) {
    if (x.layer > depth) {  // part C: the full state's own gates
      C->part_c.push_back(svp::Gate{x.kind, x.q0, (uint8_t)(x.kind == SV_CZ ? x.q1 : 0)});
      continue;
    }
    if (x.kind == SV_H && x.layer == 0) continue;  // already the leading H layer
    if (x.kind == SV_CZ && C->in_a[x.q0] != C->in_a[x.q1]) {
      const int qa = C->in_a[x.q0] ? x.q0 : x.q1, qb = C->in_a[x.q0] ? x.q1 : x.q0;
      switch (role[c++]) {
        case 0:  // P_{l} on qa (zero where x_qa != l), Z^{l} on qb (a CZ with the branch bit)
          C->ga.push_back(svp::Gate{svp::K_PEQ, (uint8_t)C->local[qa], (uint8_t)(na + jf)});
          C->gb.push_back(svp::Gate{svp::K_CZ, (uint8_t)C->local[qb], (uint8_t)(nb + jf)});
          ++jf;
          break;
        case 1:  // a sign of the output only
          C->signs.push_back({qa, qb});
          break;
        case 2: {  // projector on qa, implicit: l = x_qa; B keeps Z^{l} with its own bit
          const int bit = n_full + ja++;
          C->gb.push_back(svp::Gate{svp::K_CZ, (uint8_t)C->local[qb], (uint8_t)(nb + bit)});
          C->fix_b.push_back({bit, qa});
          break;
        }
        default: {  // projector on qb, implicit: l = x_qb; A keeps Z^{l}
          const int bit = n_full + jb++;
          C->ga.push_back(svp::Gate{svp::K_CZ, (uint8_t)C->local[qa], (uint8_t)(na + bit)});
          C->fix_a.push_back({bit, qb});
          break;
        }
      }
      continue;
    }
    std::vector<svp::Gate> &dst = C->in_a[x.q0] ? C->ga : C->gb;
    dst.push_back(svp::Gate{x.kind, (uint8_t)C->local[x.q0], (uint8_t)(x.kind == SV_CZ ? C->local[x.q1] : 0)});
  }
  return SV_OK;
}

// One half of the decomposition as a branch tree (branch-prefix sharing, §2.1: every
// branch of a half runs the same gates until its first crossing CZ).  The half's gate list
// runs on `full` (n_base + t qubits, branch bits n_base..): gates are taken in list
// order on the smallest prefix of the state that holds every branch bit touched so far
// -- the branch bits above it are still |+> (the leading H), so the state is the prefix
// times their uniform slices -- and when a gate first touches a higher branch bit the
// prefix is forked (replicated into the new slices, times 2^{-1/2} per new bit).  The
// result is the state the whole list would give on all n_base + t qubits; the work before
// each fork is done once instead of once per branch.
sv_status run_branch_tree(sv_state *full, int n_base, const std::vector<svp::Gate> &g) {
  const int n_all = full->n;
  int active = 0;  // branch bits in the prefix
  std::vector<svp::Gate> seg;
  bool first = true;
  auto flush = [&]() -> sv_status {
    if (seg.empty() && !first) return SV_OK;
    sv_state view;  // the prefix: n_base + active qubits of the same buffer
    view.n = n_base + active;
    view.psi = full->psi;
    view.owns = false;
    view.opts = full->opts;
    view.stream = full->stream;
    view.device = full->device;
    view.fresh = first;
    view.user_writes = true;
    const sv_status st = apply_gates(&view, seg);
    const sv_status werr = st == SV_OK ? take_pending_error(&view) : st;
    if (view.d_plan) cudaFree(view.d_plan);
    if (view.d_scratch) cudaFree(view.d_scratch);
    if (view.d_sums) cudaFree(view.d_sums);
    for (cudaEvent_t ev : view.events) cudaEventDestroy(ev);
    seg.clear();
    first = false;
    return werr;
  };
  for (size_t i = 0; i < g.size(); ++i) {
    const svp::Gate &x = g[i];
    // the leading H of a branch bit is what puts it in |+>: a fork does it
    if (i < (size_t)n_all && x.kind == svp::K_H && x.q0 >= n_base) continue;
    int top = -1;
    if (x.q0 >= n_base) top = x.q0 - n_base;
    if (svp::kind_two_qubit(x.kind) && x.q1 >= n_base) top = std::max(top, x.q1 - n_base);
    if (top >= active) {
      sv_status st = flush();
      if (st != SV_OK) return st;
      const cudaError_t e = svk::launch_fork(full->psi, n_base + active, n_base + top + 1, full->stream);
      if (e != cudaSuccess) { full->broken = true; return cuda_fail(e, "branch fork"); }
      active = top + 1;
    }
    seg.push_back(x);
  }
  sv_status st = flush();
  if (st != SV_OK) return st;
  if (active < n_all - n_base) {  // branch bits no gate touches: still |+>
    const cudaError_t e = svk::launch_fork(full->psi, n_base + active, n_all, full->stream);
    if (e != cudaSuccess) { full->broken = true; return cuda_fail(e, "branch fork"); }
  }
  full->fresh = false;
  full->sums_valid = false;
  return SV_OK;
}

}  // namespace

extern "C" sv_status sv_branch_counts(const sv_lattice *lat, const sv_cut *cut, int counts[5]) {
  clear_error();
  if (!lat || !cut || !counts) return fail(SV_ERR_ARG, "sv_branch_counts: NULL argument");
  if (cut->depth != 0) return fail(SV_ERR_ARG, "sv_branch_counts: cut depth must be 0");
  CutPlan C;
  sv_status st = plan_cut(lat, cut, &C);
  if (st != SV_OK) return st;
  counts[0] = C.t;
  counts[1] = C.absorbed;
  counts[2] = C.ta;
  counts[3] = C.tb;
  counts[4] = C.tf;
  return SV_OK;
}

extern "C" sv_status sv_branch_amplitudes(const sv_lattice *lat, const sv_cut *cut, const uint64_t *bits,
                                          size_t m, const sv_options *opts, double *out_re_im) {
  clear_error();
  if (!lat || !cut || (m && (!bits || !out_re_im)))
    return fail(SV_ERR_ARG, "sv_branch_amplitudes: NULL argument");
  if (cut->depth != 0)
    return fail(SV_ERR_ARG, "sv_branch_amplitudes: cut depth must be 0 (a part C needs the full state)");
  CutPlan C;
  sv_status st = plan_cut(lat, cut, &C);
  if (st != SV_OK) return st;
  const int n = C.n, na = C.na, nb = C.nb;
  for (size_t j = 0; j < m; ++j)
    if (n < 64 && (bits[j] >> n)) return fail(SV_ERR_ARG, "sv_branch_amplitudes: bitstring has bits >= n");
  sv_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  Holder A, B;
  if ((st = sv_create(na + C.ta, &o, &A.s)) != SV_OK) return st;
  if ((st = sv_create(nb + C.tb, &o, &B.s)) != SV_OK) return st;
  if ((st = run_branch_tree(A.s, na, C.ga)) != SV_OK) return st;
  if ((st = run_branch_tree(B.s, nb, C.gb)) != SV_OK) return st;
  if (m == 0) return SV_OK;
  // bitstring -> half indices, with the implicit branch bits fixed by the output bits
  std::vector<uint64_t> xab(2 * m);
  std::vector<double> sign(m, 1.0);
  for (size_t k = 0; k < m; ++k) {
    uint64_t xa = 0, xb = 0;
    for (int q = 0; q < n; ++q) {
      const uint64_t b = (bits[k] >> q) & 1ull;
      if (C.in_a[q]) xa |= b << C.local[q];
      else xb |= b << C.local[q];
    }
    for (const auto &f : C.fix_a) xa |= ((bits[k] >> f.second) & 1ull) << (na + f.first);
    for (const auto &f : C.fix_b) xb |= ((bits[k] >> f.second) & 1ull) << (nb + f.first);
    for (const auto &sg : C.signs)
      if (((bits[k] >> sg.first) & 1ull) && ((bits[k] >> sg.second) & 1ull)) sign[k] = -sign[k];
    xab[k] = xa;
    xab[m + k] = xb;
  }
  sv_state *s = A.s;
  const size_t need = 2 * m * sizeof(uint64_t) + 2 * m * sizeof(double) + 512;
  if ((st = ensure_device_buffer(&s->d_scratch, &s->d_scratch_cap, need)) != SV_OK) return st;
  uint64_t *d_x = static_cast<uint64_t *>(s->d_scratch);
  double *d_out = reinterpret_cast<double *>(static_cast<char *>(s->d_scratch) +
                                             ((2 * m * sizeof(uint64_t) + 255) & ~(size_t)255));
  // each slice carries 2^{-t_half/2}: the sum is rescaled by 2^{(ta + tb)/2}
  const double scale = std::pow(2.0, 0.5 * (C.ta + C.tb));
  cudaError_t e = cudaStreamSynchronize(B.s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_x, xab.data(), 2 * m * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = svk::launch_branch_sum(A.s->psi, na, B.s->psi, nb, C.tf, d_x, d_x + m, (int)m, scale, d_out, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_re_im, d_out, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sv_branch_amplitudes");
  for (size_t k = 0; k < m; ++k) {
    out_re_im[2 * k] *= sign[k];
    out_re_im[2 * k + 1] *= sign[k];
  }
  return SV_OK;
}

extern "C" sv_status sv_set_basis_state(sv_state *s, uint64_t x) {
  clear_error();
  if (!s) return fail(SV_ERR_ARG, "sv_set_basis_state: NULL state");
  if (s->n < 64 && (x >> s->n)) return fail(SV_ERR_ARG, "sv_set_basis_state: x has bits >= n");
  sv_status st = set_device(s);
  if (st != SV_OK) return st;
  s->sums_valid = false;
  const cudaError_t e = svk::launch_basis_state(s->psi, s->n, x, s->stream);
  if (e != cudaSuccess) { s->broken = true; return cuda_fail(e, "sv_set_basis_state"); }
  s->fresh = false;
  s->broken = false;
  if (s->prof) s->other_launches += 1;
  return SV_OK;
}

extern "C" sv_status sv_inner_product(sv_state *a, sv_state *b, double *out_re_im) {
  clear_error();
  if (!a || !b || !out_re_im) return fail(SV_ERR_ARG, "sv_inner_product: NULL argument");
  if (a->n != b->n) return fail(SV_ERR_ARG, "sv_inner_product: states of different sizes");
  if (a->device != b->device) return fail(SV_ERR_ARG, "sv_inner_product: states on different devices");
  if (a->broken || b->broken) return fail(SV_ERR_STATE, "state is unusable after an earlier failure");
  sv_status st = set_device(a);
  if (st != SV_OK) return st;
  if ((st = materialize(a)) != SV_OK) return st;
  if ((st = materialize(b)) != SV_OK) return st;
  const size_t need = (size_t)(svk::reduce_partials_needed() + 2) * 2 * sizeof(double);
  if ((st = ensure_device_buffer(&a->d_scratch, &a->d_scratch_cap, need)) != SV_OK) return st;
  double *partials = static_cast<double *>(a->d_scratch);
  double *res = partials + 2 * svk::reduce_partials_needed();
  double h[2] = {0, 0};
  // b's pending work first (the handles may use different streams)
  cudaError_t e = b->stream == a->stream ? cudaSuccess : cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = svk::launch_inner(a->psi, b->psi, a->n, partials, res, a->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, a->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(a->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sv_inner_product");
  if (a->prof) {
    a->d2h += sizeof(h);
    a->other_launches += a->n < 2 ? 1 : 2;
  }
  out_re_im[0] = h[0];
  out_re_im[1] = h[1];
  return SV_OK;
}

extern "C" sv_status sv_amplitudes_by_inner_product(const sv_lattice *lat, int split_layer, const uint64_t *bits,
                                                    size_t m, const sv_options *opts, double *out_re_im) {
  clear_error();
  if (!lat || (m && (!bits || !out_re_im))) return fail(SV_ERR_ARG, "sv_amplitudes_by_inner_product: NULL argument");
  if (split_layer < 0) return fail(SV_ERR_ARG, "sv_amplitudes_by_inner_product: split_layer must be >= 0");
  std::vector<sv_gate> g;
  sv_status st = generate(lat, &g);
  if (st != SV_OK) return st;
  const int n = lattice_qubits(lat);
  for (size_t j = 0; j < m; ++j)
    if (n < 64 && (bits[j] >> n)) return fail(SV_ERR_ARG, "sv_amplitudes_by_inner_product: bitstring has bits >= n");
  // U1 = layers 0..split_layer (the H layer included), U2 = the layers after it
  std::vector<sv_gate> g1, g2;
  for (const sv_gate &x : g) ((int)x.layer <= split_layer ? g1 : g2).push_back(x);
  sv_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  Holder A, B;
  if ((st = sv_create(n, &o, &A.s)) != SV_OK) return st;
  if ((st = sv_apply_circuit(A.s, g1.data(), g1.size())) != SV_OK) return st;  // |psi> = U1 H|0>
  if (m == 0) return SV_OK;
  if ((st = sv_create(n, &o, &B.s)) != SV_OK) return st;
  std::vector<svp::Gate> g2_inv;
  if ((st = convert_gates(n, g2.data(), g2.size(), true, &g2_inv)) != SV_OK) return st;
  for (size_t j = 0; j < m; ++j) {
    // |phi_x> = U2^dagger |x>;  alpha_x = <phi_x|psi>: on plan kernels the last pass of
    // phi_x sums the inner product instead of storing phi_x
    if ((st = sv_set_basis_state(B.s, bits[j])) != SV_OK) return st;
    bool fused = false;
    if ((st = apply_gates_inner(B.s, g2_inv, A.s, out_re_im + 2 * j, &fused)) != SV_OK) return st;
    if (fused) continue;
    if ((st = sv_apply_circuit_inverse(B.s, g2.data(), g2.size())) != SV_OK) return st;
    if ((st = sv_inner_product(B.s, A.s, out_re_im + 2 * j)) != SV_OK) return st;
  }
  return SV_OK;
}

extern "C" sv_status sv_branch_full_state(const sv_lattice *lat, const sv_cut *cut, const sv_options *opts,
                                          sv_state *out) {
  clear_error();
  if (!lat || !cut || !out) return fail(SV_ERR_ARG, "sv_branch_full_state: NULL argument");
  CutPlan C;
  sv_status st = plan_cut(lat, cut, &C, false);
  if (st != SV_OK) return st;
  if (out->n != C.n) return fail(SV_ERR_ARG, "sv_branch_full_state: output state has the wrong size");
  if (cut->half_a_mask != (C.na >= 64 ? ~0ull : (1ull << C.na) - 1))
    return fail(SV_ERR_ARG, "sv_branch_full_state: half A must be qubits 0..n_A-1");
  if (out->broken) return fail(SV_ERR_STATE, "state is unusable after an earlier failure");
  sv_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  Holder A, B;
  if ((st = sv_create(C.na + C.ta, &o, &A.s)) != SV_OK) return st;
  if ((st = sv_create(C.nb + C.tb, &o, &B.s)) != SV_OK) return st;
  if ((st = run_branch_tree(A.s, C.na, C.ga)) != SV_OK) return st;
  if ((st = run_branch_tree(B.s, C.nb, C.gb)) != SV_OK) return st;
  if ((st = set_device(out)) != SV_OK) return st;
  cudaError_t e = cudaStreamSynchronize(A.s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B.s->stream);
  // each branch slice carries 2^{-t/2} per half
  const float scale = std::ldexp(1.0f, C.tf);
  // the tensor-core precisions: the product on tcgen05 (TF32x3), else on the CUDA cores
  const bool tc = (o.precision == SV_PREC_TF32X3 || o.precision == SV_PREC_F16X3) &&
                  svk::fused_supported() && svk::outer_sum_tc_supported(C.na, C.nb, C.tf);
  void *scratch = nullptr;
  int *d_err = nullptr;
  if (e == cudaSuccess && tc) {
    e = cudaMalloc(&scratch, svk::outer_sum_tc_scratch(C.na, C.nb, C.tf) + 256);
    if (e == cudaSuccess) {
      d_err = reinterpret_cast<int *>(static_cast<char *>(scratch) + svk::outer_sum_tc_scratch(C.na, C.nb, C.tf));
      e = cudaMemsetAsync(d_err, 0, sizeof(int), out->stream);
    } else {
      scratch = nullptr;
    }
    if (e == cudaSuccess) {
      profile_begin(out);
      e = svk::launch_outer_sum_tc(A.s->psi, C.na, B.s->psi, C.nb, C.tf, scale, out->psi, scratch, d_err, out->stream);
      profile_end(out, std::ldexp(8.0, C.n));
    }
  } else if (e == cudaSuccess) {
    profile_begin(out);
    e = svk::launch_outer_sum(A.s->psi, C.na, B.s->psi, C.nb, C.tf, scale, out->psi, out->stream);
    profile_end(out, std::ldexp(8.0, C.n));
  }
  int h_err = 0;
  if (d_err && e == cudaSuccess) {
    e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, out->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(out->stream);
  }
  if (scratch) cudaFree(scratch);
  out->sums_valid = false;
  if (e != cudaSuccess) { out->broken = true; return cuda_fail(e, "sv_branch_full_state"); }
  if (h_err) { out->broken = true; return fail(SV_ERR_TIMEOUT, "sv_branch_full_state: a tensor-core wait gave up"); }
  out->fresh = false;
  if (out->prof) out->other_launches += 1;
  // the crossing CZs taken as output signs act on the product state like any CZ
  // (they commute with part C: neither qubit meets a non-diagonal gate after them)
  std::vector<svp::Gate> signs;
  for (const auto &sg : C.signs) signs.push_back(svp::Gate{svp::K_CZ, (uint8_t)sg.first, (uint8_t)sg.second});
  if (!signs.empty() && (st = apply_gates(out, signs)) != SV_OK) return st;
  // part C (Eq. 3): the layers after the cut depth on the reconstructed state
  if (!C.part_c.empty() && (st = apply_gates(out, C.part_c)) != SV_OK) return st;
  e = cudaStreamSynchronize(out->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sv_branch_full_state");
  return SV_OK;
}
