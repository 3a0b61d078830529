"""Plant plausible mistakes in copies of the oracle (CPU only) and check the pins catch each.

Every mutation is a one-token change of the kind a careful reader could still
miss: a dropped term, a wrong sign, a wrong index, a transposed operand, a
swapped pair.  A copy of gcnn_oracle.c is edited in a temporary directory and
built there; the committed oracle is never modified.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "gcnn_oracle.c")

MUTATIONS = {
    "std_drops_eps": ("sqrt((var > 0.0 ? var : 0.0) + n->eps)", "sqrt((var > 0.0 ? var : 0.0))"),
    "std_grad_sign": ("(v - mean) / (d * sd)", "(mean - v) / (d * sd)"),
    "msg_source_block": ("msg_w[(int64_t)(k - H) * 2 * H + H + c]", "msg_w[(int64_t)(k - H) * 2 * H + c]"),
    "update_transposed": ("acc += u[k] * w->upd_w[(int64_t)k * H + c]", "acc += u[k] * w->upd_w[(int64_t)c * 16 * H + k]"),
    "scalers_swapped": ("s == 1 ? (double)n->amp[i] : (double)n->att[i]", "s == 1 ? (double)n->att[i] : (double)n->amp[i]"),
    "sum_pool": ("s / (double)(b - a) : 0.0", "s : 0.0"),
    "max_ties_not_shared": ("da[3 * H + c] / nmax", "da[3 * H + c]"),
    "adam_bias_b1_for_b2": ("c2 = 1.0 - pow(b2", "c2 = 1.0 - pow(b1"),
    "rows_sorted_descending": ("col[b] > v", "col[b] < v"),
    "rev_self": ("if (col[q] == (int32_t)i) { rev[p] = q; break; }", "if (col[q] == (int32_t)i) { rev[p] = p; break; }"),
    "mean_off_by_one": ("double mean = sum / d;", "double mean = sum / (d + 1.0);"),
    "amp_log_d": ("amp[i] = (float)(log(d + 1.0) / delta);", "amp[i] = (float)(log(d) / delta);"),
    "head_no_relu": ("out += (acc > 0.0 ? acc : 0.0) * w2[c];", "out += acc * w2[c];"),
    "msg_bwd_source_uses_dest_weights": ("wm(&n, w.msg_w, H + k, c) * dm", "wm(&n, w.msg_w, k, c) * dm"),
    "pool_bwd_no_division": ("dx[i * H + k] = dg[g * H + k] / (double)(b - a);", "dx[i * H + k] = dg[g * H + k];"),
    "min_ties_counted_as_max": ("nmin += (v == mn);", "nmin += (v == mx);"),
    "bond_message_feature_index": ("(double)n->eattr[(int64_t)e * n->F + f]", "(double)n->eattr[(int64_t)e * n->F]"),
    "bond_grad_feature_index": ("(double)eattr[e * F + fi] * dm[e * H + c]", "(double)eattr[e * F] * dm[e * H + c]"),
    "bond_attr_in_store_order": ("eattr[p * F + f] = st_eattr[pos_sid[p] * F + f];",
                                 "eattr[p * F + f] = st_eattr[p * F + f];"),
    "bond_attr_left_behind_by_sort": ("col[b + 1] = col[b]; pos_sid[b + 1] = pos_sid[b]; --b;",
                                      "col[b + 1] = col[b]; --b;"),
    "node_loss_over_graphs": ("dpredn[i] = N > 0 ? node_weight * 2.0 * r / (double)N : 0.0;",
                              "dpredn[i] = N > 0 ? node_weight * 2.0 * r / (double)G : 0.0;"),
    "node_head_no_relu": ("out += (z > 0.0 ? z : 0.0) * w2[c];", "out += z * w2[c];"),
    "node_head_grad_not_into_trunk": ("dx[i * H + k] += w1[(int64_t)k * Hh + c] * dz;", ";"),
}


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, workdir, monkeypatch):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor not unique/present: {old!r}"
    path = os.path.join(workdir, f"{name}.c")
    with open(path, "w") as f:
        f.write(text.replace(old, new))
    so = os.path.join(workdir, f"lib{name}.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-o", so, path, "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle.load(so))
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            if pin is oracle_pins.pin_finite_differences:
                pin(n_coords=60)
            else:
                pin()
        except (AssertionError, MemoryError, ValueError, IndexError):
            caught.append(pin.__name__)
    assert caught, f"no pin catches the planted mistake {name}"
