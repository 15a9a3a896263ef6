"""Mutation tests of the oracle's pins.

The oracle is only as good as the checks that tie it to the paper and to the
mathematics.  Each case below plants one plausible mistake in a copy of the C
oracle (a dropped term, a wrong sign, comparison or index, a transposed
operand, a swapped tie-break), compiles the copy, and runs the CPU pin suite
(`tests/test_oracle.py`) against it.  The pins must reject every mutant: a
mutant that passes marks a mistake the pins would not have caught.

The originals are matched as exact text and must occur once in the source, so
a refactor of the oracle that moves one of them fails here loudly instead of
silently testing nothing.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_SRC = os.path.join(ROOT, "oracle", "kdt_oracle.c")

# name -> list of (original text, mutated text); each names the part of the
# method it breaks
MUTANTS = {
    # builder: left-subtree size of the complete tree (level order, Sec. 3)
    "left_size_off_by_one": [(
        "return (half - 1) + (last < half ? last : half);",
        "return half + (last < half ? last : half);")],
    # builder: round-robin split dimension taken one level late
    "split_dim_next_level": [(
        "orc_widest_dim(pts, D, S, n) : orc_level(node) % D;",
        "orc_widest_dim(pts, D, S, n) : orc_level(node + 1) % D;")],
    # builder: tie-break on the input index reversed
    "sort_tie_reversed": [(
        "return (ia > ib) - (ia < ib);",
        "return (ia < ib) - (ia > ib);")],
    # builder: the classic median instead of the left-balanced rank
    "median_not_left_balanced": [(
        "node_pid[node] = S[L];",
        "node_pid[node] = S[n / 2];")],
    # builder: children written to each other's slots
    "children_swapped": [
        ("orc_build_rec(pts, N, D, S, L, 2 * node + 1, node_pid, node_dim)",
         "orc_build_rec(pts, N, D, S, L, 2 * node + 2, node_pid, node_dim)"),
        ("orc_build_rec(pts, N, D, S + L + 1, n - L - 1, 2 * node + 2, node_pid, node_dim)",
         "orc_build_rec(pts, N, D, S + L + 1, n - L - 1, 2 * node + 1, node_pid, node_dim)")],
    # widest-extent builder: ties go to the highest dimension
    "widest_tie_high": [(
        "if (ext > best_ext) {",
        "if (ext >= best_ext) {")],
    # distance: the last coordinate's term dropped
    "d2_drops_last_term": [(
        "    for (int j = 1; j < D; ++j) {\n        float dj = p[j] - q[j];",
        "    for (int j = 1; j < D - 1; ++j) {\n        float dj = p[j] - q[j];")],
    # distance: the first term not squared
    "d2_first_term_unsquared": [(
        "float s = diff * diff;",
        "float s = diff;")],
    # k-best list: ties on d2 go to the larger id
    "pair_tie_larger_id": [(
        "    return ia < ib;\n}",
        "    return ia > ib;\n}")],
    # processNode: the radius test exclusive
    "accept_exclusive": [(
        "if (!(d2 <= L->r2))",
        "if (!(d2 < L->r2))")],
    # the cull radius never shrinks (results unchanged, visits not)
    "cull_never_shrinks": [(
        "return L->count == L->k ? L->d2[L->k - 1] : L->r2;",
        "return L->r2;")],
    # plain definition: the radius used unsquared
    "brute_radius_unsquared": [(
        "    float r2 = max_radius * max_radius;\n    float *ld",
        "    float r2 = max_radius;\n    float *ld")],
    # tree traversals: the radius used unsquared
    "tree_radius_unsquared": [(
        "orc_list L = {k, 0, max_radius * max_radius, ld, li};",
        "orc_list L = {k, 0, max_radius, ld, li};")],
    # FP64 brute force: ties to the larger index
    "f64_tie_larger_id": [(
        "if (count == k && !(s < od[k - 1] || (s == od[k - 1] && i < oi[k - 1])))",
        "if (count == k && !(s < od[k - 1] || (s == od[k - 1] && i > oi[k - 1])))")],
    # recursion: the far child entered before the close child
    "rec_far_first": [
        ("        orc_rec(T, close_child);\n",
         "        orc_rec(T, far_child);\n"),
        ("            orc_rec(T, far_child);\n",
         "            orc_rec(T, close_child);\n")],
    # stack-free machine: the close side flips on sd == 0
    "stackfree_close_side_ge": [(
        "int64_t first = T->ordered && sd > 0.0f ? right : left;",
        "int64_t first = T->ordered && sd >= 0.0f ? right : left;")],
    # stack-free machine: the second child taken as the right one always
    "stackfree_second_always_right": [(
        "int64_t second = first == left ? right : left;",
        "int64_t second = right;")],
    # stack-free machine: the cull test exclusive
    "stackfree_cull_exclusive": [(
        "return query_side || sd * sd <= orc_list_cull(T->L);",
        "return query_side || sd * sd < orc_list_cull(T->L);")],
    # stack-free machine: the query's side of the plane swapped
    "stackfree_side_swapped": [(
        "int query_side = child == left ? sd <= 0.0f : sd > 0.0f;",
        "int query_side = child == left ? sd > 0.0f : sd <= 0.0f;")],
    # stack-free machine: the root's parent index (C division rounds -1/2 to 0)
    "stackfree_parent_formula": [(
        "int64_t up = at == 0 ? -1 : (at - 1) / 2;",
        "int64_t up = (at - 1) / 2;")],
    # stack-free machine: back from the second child read as back from the first
    "stackfree_arrival_second": [(
        "(from == first ? ORC_FROM_FIRST : ORC_FROM_SECOND)",
        "(from == second ? ORC_FROM_FIRST : ORC_FROM_SECOND)")],
    # close-first machine: processing on arrival switched off for the wrong
    # variant.  (Judging the far child against the radius from before the
    # node was processed is not a mistake a pin can catch: the node lies on
    # its own splitting plane, so its distance is at least fl(sd^2), and
    # accepting it never shrinks the radius below fl(sd^2).)
    "close_first_flag_typo": [(
        "            if (T->ordered != 2)\n                orc_process(T, at);",
        "            if (T->ordered != 1)\n                orc_process(T, at);")],
    # stack-free machine: a child needs the query on its side (no overlap test)
    "stackfree_no_overlap": [(
        "return query_side || sd * sd <= orc_list_cull(T->L);",
        "return query_side;")],
    # stack-free machine: no step from the first child to the second one
    "stackfree_skips_second_after_first": [(
        "            if (orc_enters(T, second, left, sd))\n                next = second;\n            break;\n"
        "        default:",
        "            break;\n        default:")],
    # learned-radius feature: the descent goes to the far child
    "descent_far_child": [(
        "int64_t child = 2 * node + 1 + (sd > 0.0f);",
        "int64_t child = 2 * node + 1 + (sd <= 0.0f);")],
    # bfloat16 rounding: ties away from zero instead of to even
    "bf16_ties_away": [(
        "u = u + 0x7FFFu + lsb;",
        "u = u + 0x8000u;")],
    # MLP forward: an extra ReLU on the output
    "mlp_output_relu": [(
        "            o += w3[i] * h2[i];\n        y[s] = o;",
        "            o += w3[i] * h2[i];\n        y[s] = o > 0.0 ? o : 0.0;")],
    # MLP backward: the loss derivative without its factor 2
    "grad_loss_factor": [(
        "double go = 2.0 * e / (double)n;",
        "double go = e / (double)n;")],
    # MLP backward: the second ReLU's mask dropped
    "grad_relu_mask_dropped": [(
        "g2[i] = z2[i] > 0.0 ? go * w3[i] : 0.0;",
        "g2[i] = go * w3[i];")],
    # MLP backward: W2 transposed in the back-propagation
    "grad_w2_transposed": [(
        "a += W2[(int64_t)i * H + j] * g2[i];",
        "a += W2[(int64_t)j * H + i] * g2[i];")],
    # MLP backward: the first layer's input index swapped for the row
    "grad_w1_input_index": [(
        "gW1[i * 4 + j] += g1[i] * xs[j];",
        "gW1[i * 4 + j] += g1[i] * xs[3 - j];")],
    # range machine: the ball test exclusive
    "range_ball_exclusive": [(
        "hit = v <= r2;",
        "hit = v < r2;")],
    # range machine: the box's left-subtree test exclusive (misses points
    # equal to the split coordinate, which ties can put on the left)
    "range_box_left_exclusive": [(
        "left_in = a[dim] <= split;",
        "left_in = a[dim] < split;")],
    # range machine: the ball's right-subtree overlap test dropped
    "range_ball_right_no_overlap": [(
        "right_in = sd > 0.0f || sd * sd <= r2;",
        "right_in = sd > 0.0f;")],
    # payload reductions: the mean divides by one more than the count
    "reduce_mean_count": [(
        "s = s / (float)n;",
        "s = s / (float)(n + 1);")],
    # payload reductions: the density over pi * R instead of pi * R^2
    "reduce_density_unsquared": [(
        "s = s / (ORC_PI_F * R2);",
        "s = s / (ORC_PI_F * sqrtf(R2));")],
    # tree level off by one below the root (builder and traversals agree with
    # each other, so only the pins on the tree itself can see it)
    "level_formula": [(
        "    while (v > 1) {",
        "    while (v > 2) {")],
    # widest-extent builder: the upper end of the extent never grows
    "widest_extent_upper_end": [(
        "            if (v > hi)",
        "            if (v < hi)")],
    # recursion, unordered: the right child needs the query on its side
    "rec_unordered_right_no_overlap": [(
        "if (sd > 0.0f || sd * sd <= orc_list_cull(T->L)) {",
        "if (sd > 0.0f) {")],
    # learned-radius feature: the descent splits every level in dimension 0
    "descent_dim_zero": [(
        "        int dim = node_dim ? node_dim[node] : orc_level(node) % D;",
        "        int dim = node_dim ? node_dim[node] : 0;")],
    # learned-radius feature on stored-split trees: the stored dimension ignored
    "descent_ignores_stored_dim": [(
        "        int dim = node_dim ? node_dim[node] : orc_level(node) % D;",
        "        int dim = orc_level(node) % D;")],
    # learned-radius feature on stored-split trees: the parent's dimension read
    "descent_stored_dim_of_parent": [(
        "        int dim = node_dim ? node_dim[node] : orc_level(node) % D;",
        "        int dim = node_dim ? node_dim[node ? (node - 1) / 2 : 0] : orc_level(node) % D;")],
    # result emission: empty slots marked with id 0
    "empty_slot_id_zero": [(
        "            ids[i] = -1;\n            d2[i] = INFINITY;\n        }\n    }\n}",
        "            ids[i] = 0;\n            d2[i] = INFINITY;\n        }\n    }\n}")],
    # MLP forward: the first layer's bias dropped
    "mlp_forward_b1_dropped": [(
        "        for (int i = 0; i < H; ++i) {\n            double a = b1[i];\n            for (int j = 0; j < 4; ++j)\n"
        "                a += W1[i * 4 + j] * xs[j];\n            h1[i] = a > 0.0 ? a : 0.0;",
        "        for (int i = 0; i < H; ++i) {\n            double a = 0.0;\n            for (int j = 0; j < 4; ++j)\n"
        "                a += W1[i * 4 + j] * xs[j];\n            h1[i] = a > 0.0 ? a : 0.0;")],
    # MLP loss: the sum not divided by the sample count
    "mlp_loss_not_mean": [(
        "return loss / (double)n;",
        "return loss;")],
    # MLP backward: the first bias takes the second layer's gradient
    "grad_b1_from_layer2": [(
        "gb1[i] += g1[i];",
        "gb1[i] += g2[i];")],
    # ball definition: exclusive radius
    "radius_brute_exclusive": [(
        "            if (v <= r2) {",
        "            if (v < r2) {")],
    # box definition: exclusive upper corner
    "box_brute_upper_exclusive": [(
        "if (!(lo[q * D + j] <= v && v <= hi[q * D + j])) {",
        "if (!(lo[q * D + j] <= v && v < hi[q * D + j])) {")],
    # range machine: the box's right-subtree test exclusive
    "range_box_right_exclusive": [(
        "right_in = b[dim] >= split;",
        "right_in = b[dim] > split;")],
    # range machine: hit distances not stored
    "range_d2_not_stored": [(
        "                        d2[count] = v;\n",
        "                        d2[count] = 0.0f;\n")],
    # payload reductions: no special case for an empty hit set
    "reduce_empty_not_zero": [(
        "        if (n == 0)\n            s = 0.0f;\n        else if (mode == 1)",
        "        if (mode == 1)")],
    # kNN reductions: the empty slots counted as neighbours
    "knn_reduce_counts_empty": [(
        "while (n < k && ids[q * k + n] >= 0)",
        "while (n < k && ids[q * k + n] >= -1)")],
    # widest-extent builder: the extent taken as the upper end alone
    "widest_extent_not_difference": [(
        "        float ext = hi - lo;",
        "        float ext = hi;")],
    # k-best list: the "greater" branch of the pair order dropped
    "pair_less_missing_branch": [(
        "    if (db < da)\n        return 0;\n",
        "")],
    # recursion, unordered: the left child needs the query on its side
    "rec_unordered_left_no_overlap": [(
        "if (sd <= 0.0f || sd * sd <= orc_list_cull(T->L)) {",
        "if (sd <= 0.0f) {")],
    # unordered machine: from the parent, the second (right) child is never
    # taken when the first one is out of range
    "unordered_from_parent_skips_second": [(
        "            else if (orc_enters(T, second, left, sd))\n                next = second;\n",
        "")],
    # learned-radius feature: the descent stops one node early
    "descent_stops_early": [(
        "        if (child >= N)\n            break;",
        "        if (child >= N - 1)\n            break;")],
    # bfloat16 rounding: the tie-breaking bit taken one place too low
    "bf16_lsb_position": [(
        "uint32_t lsb = (u >> 16) & 1u;",
        "uint32_t lsb = (u >> 15) & 1u;")],
    # MLP backward: W2's gradient against the pre-activations
    "grad_w2_preactivation": [(
        "gW2[(int64_t)i * H + j] += g2[i] * h1[j];",
        "gW2[(int64_t)i * H + j] += g2[i] * z1[j];")],
    # forward bound: the bfloat16 unit roundoff taken as 2^-9
    "bound_bf16_roundoff_halved": [(
        "const double ub = 1.0 / 256.0;",
        "const double ub = 1.0 / 512.0;")],
    # forward bound: layer 1's error not carried through the hidden contraction
    "bound_no_propagation_layer2": [(
        "                prop += fabs(w) * e1[i];\n",
        "")],
    # forward bound: the output layer's error from the hidden layer dropped
    "bound_no_propagation_output": [(
        "            prop += fabs(w3[j]) * e2[j];\n",
        "")],
    # forward bound: the FP32 allowance of layer 1 dropped
    "bound_layer1_fp32_dropped": [(
        "            e1[i] = ub * (h1[i] + g1 * S) + g1 * S;",
        "            e1[i] = ub * h1[i];")],
    # gradient bound: a pre-activation within its bound of 0 not treated as switchable
    "grad_bound_no_mask_flip": [(
        "            const double dg2 = amb ? M2 : (z2[i] > 0.0 ? (dgo + uf * ago) * fabs(w3[i]) : 0.0);",
        "            const double dg2 = z2[i] > 0.0 ? (dgo + uf * ago) * fabs(w3[i]) : 0.0;")],
    # gradient bound: the bfloat16 rounding of the back-propagated operand dropped
    "grad_bound_no_g2_rounding": [(
        "            dg2b[i] = dg2 + ub * M2;",
        "            dg2b[i] = dg2;")],
    # gradient bound: the activation error not carried into the weight gradient
    "grad_bound_no_h1_error_in_dw2": [(
        "acc[(bW2 - bound) + (int64_t)i * H + j] += dg2b[i] * (h1[j] + e1[j]) + M2b[i] * e1[j];",
        "acc[(bW2 - bound) + (int64_t)i * H + j] += dg2b[i] * h1[j];")],
    # gradient bound: the output error not carried into go
    "grad_bound_no_output_error": [(
        "        const double de = e3 + uf * (fabs(err) + e3);",
        "        const double de = uf * fabs(err);")],
    # payload reductions: the payload row stride dropped
    "reduce_payload_stride": [(
        "s = s + payload[(int64_t)hits[i] * C + c];",
        "s = s + payload[(int64_t)hits[i] + c];")],
    # kNN reductions: the output row stride off by one
    "knn_reduce_output_stride": [(
        "orc_reduce_one(payload, C, ids + q * k, n, mode, R2, out + q * C);",
        "orc_reduce_one(payload, C, ids + q * k, n, mode, R2, out + q * (C > 1 ? C - 1 : C));")],
    # kNN reductions: the disc through the nearest neighbour, not the farthest
    "knn_reduce_nearest_disc": [(
        "float R2 = n ? d2[q * k + n - 1] : 0.0f;",
        "float R2 = n ? d2[q * k] : 0.0f;")],
}


def _mutated_source(src, edits):
    for old, new in edits:
        assert src.count(old) == 1, f"mutation target not found exactly once: {old!r}"
        src = src.replace(old, new)
    return src


def test_mutation_targets_are_unique():
    src = open(ORACLE_SRC).read()
    for name, edits in MUTANTS.items():
        out = _mutated_source(src, edits)
        assert out != src, name


def _run_pins(name, src, workdir):
    """Compile one copy of the oracle and run the pin suite against it;
    returns (name, pytest's exit status or None, the end of its output)."""
    d = os.path.join(workdir, name)
    os.makedirs(d)
    c_path = os.path.join(d, "kdt_oracle.c")
    with open(c_path, "w") as f:
        f.write(src)
    # built here, so that a mutant that does not compile is reported as such
    # rather than counted as caught by the pins
    cc = subprocess.run(["gcc", *oracle.CFLAGS, "-o", os.path.join(d, "libkdt_oracle.so"), c_path, "-lm"],
                        capture_output=True, text=True)
    if cc.returncode != 0:
        return name, "compile", cc.stderr.strip()[-400:]
    env = dict(os.environ, KDT_ORACLE_SRC=c_path)
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle.py"), "-x", "-q",
           "-p", "no:cacheprovider", "-m", "not gpu"]
    try:
        r = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return name, None, "timed out"
    tail = "\n".join((r.stdout + r.stderr).strip().splitlines()[-3:])
    return name, r.returncode, tail


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_pins_reject_every_mutant(tmp_path):
    src = open(ORACLE_SRC).read()
    # the unmutated copy must pass, or every "rejection" below means nothing
    name, rc, tail = _run_pins("unmutated", src, str(tmp_path))
    assert rc == 0, f"the pin suite fails on an unmutated copy of the oracle:\n{tail}"
    jobs = [(n, _mutated_source(src, e)) for n, e in MUTANTS.items()]
    workers = max(1, min(8, (os.cpu_count() or 1)))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda j: _run_pins(j[0], j[1], str(tmp_path)), jobs))
    broken = [(n, tail) for n, rc, tail in results if rc == "compile"]
    assert not broken, "mutants that do not compile:\n" + "\n".join(f"  {n}: {t}" for n, t in broken)
    survivors = [(n, tail) for n, rc, tail in results if rc == 0]
    assert not survivors, "mutants the oracle pins do not catch:\n" + "\n".join(
        f"  {n}: {t}" for n, t in survivors)
