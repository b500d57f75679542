"""The oracle's pins catch plausible mistakes (no GPU).

Each case plants one mistake in the oracle, on the CPU and only for the duration of the test (a
dropped term, a wrong sign, a wrong factor, a skipped step), then runs the pins that guard that
part of the oracle and requires at least one of them to fail. A mistake no pin notices would mean
the oracle is pinned to itself there.
"""
import numpy as np
import pytest

import netgen
from oracle import companion as cm
from oracle import dense
from oracle import emt
from oracle import hinv
from oracle import modify
from oracle import partition as pt
from tests import test_oracle as T


def _tile():
    return emt.Network(netgen.tile(1_000_000), T.DT, levels=2)


def _some_pin_fails(pins):
    for pin in pins:
        try:
            pin()
        except Exception:   # an assertion, or arithmetic that broke down under the mistake
            return True
    return False


def _patch_elements(monkeypatch, change):
    orig = cm.elements

    def mutated(net, dt):
        el = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in orig(net, dt).items()}
        change(net, el)
        return el

    monkeypatch.setattr(cm, "elements", mutated)


def test_rc_history_with_the_wrong_sign_is_caught(monkeypatch):
    def change(net, el):
        nb = el["n_series"]
        rc = np.zeros(len(el["beta"]), bool)
        rc[:nb] = np.asarray(net["kind"]) == cm.KIND_RC
        el["beta"][rc] *= -1.0

    _patch_elements(monkeypatch, change)
    assert _some_pin_fails([T.test_rc_series_sine_steady_state_bilinear, T.test_passivity_sources_off,
                            T.test_lossless_lc_network_conserves_energy_exactly])


def test_rl_conductance_with_l_over_dt_is_caught(monkeypatch):
    def change(net, el):
        nb = el["n_series"]
        for e in range(nb):
            if net["kind"][e] == cm.KIND_RL:
                x = float(net["L"][e]) / T.DT   # should be 2L/dt
                g = 1.0 / (float(net["R"][e]) + x)
                el["g"][e], el["alpha"][e], el["beta"][e] = g, g, g * (x - float(net["R"][e]))

    _patch_elements(monkeypatch, change)
    assert _some_pin_fails([T.test_rl_sine_steady_state_bilinear])


def test_dropped_to_bus_history_term_is_caught(monkeypatch):
    def mutated(el, Ih, n_bus):
        i = np.zeros(n_bus)
        np.add.at(i, el["a"], -Ih)   # the +I_h at the to-bus is missing
        return i

    monkeypatch.setattr(cm, "history_injection", mutated)
    assert _some_pin_fails([T.test_kirchhoff_balance_every_step, T.test_rl_sine_steady_state_bilinear])


def test_paper_core_as_identity_is_caught(monkeypatch):
    orig = hinv.HInv._build_node

    def mutated(self, p):
        orig(self, p)
        if self.mode == hinv.PAPER and p in self.C:
            self.C[p] = np.eye(self.C[p].shape[0])   # should be [[0, I], [I, 0]]

    monkeypatch.setattr(hinv.HInv, "_build_node", mutated)
    nw = _tile()
    assert _some_pin_fails([T.test_two_bus_golden, lambda: T.test_eq5_offdiagonal_blocks_vanish(nw),
                            lambda: T.test_paper_store_equals_dense_algorithm1(nw)])


def test_cut_columns_with_plus_g_are_caught(monkeypatch):
    orig = hinv.HInv.cut_columns

    def mutated(self, p):
        hl, hr = orig(self, p)
        return -hl, hr

    monkeypatch.setattr(hinv.HInv, "cut_columns", mutated)
    nw = _tile()
    assert _some_pin_fails([T.test_two_bus_golden, lambda: T.test_exact_store_equals_dense_inverse(nw)])


def test_exact_core_without_the_swap_term_is_caught(monkeypatch):
    orig = hinv.HInv._build_node

    def mutated(self, p):
        orig(self, p)
        if self.mode == hinv.EXACT and p in self.C:
            k = self.P[p].shape[1]
            hl, hr = self.hl[p], self.hr[p]
            S = np.block([[hl.T @ self.P[p], np.zeros((k, k))], [np.zeros((k, k)), hr.T @ self.Q[p]]])
            self.C[p] = np.linalg.pinv(S + 1e-3 * np.eye(2 * k))   # S lost its X = [[0, I], [I, 0]]

    monkeypatch.setattr(hinv.HInv, "_build_node", mutated)
    nw = _tile()
    assert _some_pin_fails([lambda: T.test_exact_store_equals_dense_inverse(nw),
                            T.test_no_coupling_paper_equals_exact])


def test_sherman_morrison_with_the_wrong_denominator_is_caught(monkeypatch):
    def mutated(Ginv, u, delta):
        z = Ginv @ u
        d = 1.0 - delta * float(u @ z)   # should be 1 + delta u^T z
        return Ginv - (delta / d) * np.outer(z, z)

    monkeypatch.setattr(dense, "sherman_morrison", mutated)
    nw = _tile()
    assert _some_pin_fails([lambda: T.test_sherman_morrison_and_woodbury_closed_forms(nw)])


def test_algorithm2_without_the_leaf_reinversion_is_caught(monkeypatch):
    orig = modify.touched_path

    def mutated(tree, a_pos, b_pos, to_root):
        leaves, order, top = orig(tree, a_pos, b_pos, to_root)
        return [], order, top   # the touched leaves keep their old inverses

    monkeypatch.setattr(modify, "touched_path", mutated)
    nw = _tile()
    assert _some_pin_fails([lambda: T.test_algorithm2_to_root_equals_rebuild(nw)])


def test_lca_one_level_too_high_is_caught(monkeypatch):
    orig = pt.lca

    def mutated(tree, u, v):
        w = orig(tree, u, v)
        p = int(tree["parent"][w])
        return p if p >= 0 else w

    monkeypatch.setattr(pt, "lca", mutated)
    assert _some_pin_fails([T.test_lca_brute_force])


def test_coupled_admittance_with_the_wrong_mutual_sign_is_caught(monkeypatch):
    orig = cm.coupled_rl_admittance
    monkeypatch.setattr(cm, "coupled_rl_admittance", lambda R, L, M, dt: orig(R, L, -M, dt))
    assert _some_pin_fails([T.test_coupled_rl_admittance_closed_form,
                            T.test_three_phase_balanced_steady_state_uses_positive_sequence_inductance])


def test_bisection_without_kernighan_lin_is_caught(monkeypatch):
    monkeypatch.setattr(pt, "_kl", lambda side, nbr, wt, passes=4: side.copy())
    pins = [lambda g=g: T.test_bisection_reaches_brute_force_minimum(*g) for g in (
        ("path", T._graph_path(11), 11), ("cycle", T._graph_cycle(12), 12),
        ("barbell", T._graph_barbell(6), 12), ("ladder", T._graph_ladder(6), 12))]
    assert _some_pin_fails(pins + [T.test_kl_never_worse_than_growth_and_small_brute_force])


def test_three_phase_sources_with_the_wrong_sequence_are_caught(monkeypatch):
    from oracle import emt3
    monkeypatch.setattr(emt3, "phase_shift", lambda p: 2.0 * np.pi * p / 3.0)   # a-c-b instead of a-b-c
    assert _some_pin_fails([T.test_three_phase_stepping_without_mutual_is_three_shifted_single_phase_runs,
                            T.test_three_phase_balanced_steady_state_uses_positive_sequence_inductance])


def test_fault_clearing_by_restoring_the_pre_fault_solver_is_caught(monkeypatch):
    # the reading that clearing a fault puts back G and the solver saved when it came on, which
    # also undoes every change made in between
    saved = {}
    orig_change = emt._Solver.change

    def change(self, a, b, delta):
        if b < 0 and delta > 0:
            saved.setdefault(id(self), {})[a] = (self.G.copy(), self.s)
        if b < 0 and delta < 0 and a in saved.get(id(self), {}):
            self.G, self.s = saved[id(self)].pop(a)
            return
        orig_change(self, a, b, delta)

    monkeypatch.setattr(emt._Solver, "change", change)
    assert _some_pin_fails([lambda: T.test_kirchhoff_balance_through_trips_and_overlapping_faults("dense")])


def test_block_cut_columns_without_the_cross_phase_entries_are_caught(monkeypatch):
    # the node-level reading carried into block cuts: only the same-phase vertex of the left bus
    orig = hinv.HInv.cut_columns

    def mutated(self, p):
        hl, hr = orig(self, p)
        if int(self.tree.get("cut_w", 1)) == 3:
            lo = int(self.tree["lo"][int(self.tree["left"][p])])
            ro = int(self.tree["lo"][int(self.tree["right"][p])])
            rows = np.arange(hl.shape[0])[:, None] + lo
            cols = (np.argmax(hr, axis=0) + ro)[None, :]
            hl = np.where(rows % 3 == cols % 3, hl, 0.0)
        return hl, hr

    monkeypatch.setattr(hinv.HInv, "cut_columns", mutated)
    assert _some_pin_fails([T.test_block_tree_keeps_buses_together_and_factors_each_h_exactly,
                            T.test_block_store_is_the_exact_inverse_and_paper_store_is_algorithm1])


def test_block_tree_with_a_dropped_bus_pair_is_caught(monkeypatch):
    orig = pt.build_block_tree

    def mutated(*a, **k):
        t = dict(orig(*a, **k))
        B = int(t["cut_w"])
        e0, e1 = int(t["cut_ptr"][0]), int(t["cut_ptr"][1])
        keep = np.ones(len(t["cut_b"]), bool)
        keep[e1 - B:e1] = False   # the root's last joined bus pair is lost
        t["cut_b"] = t["cut_b"][keep]
        t["cut_e"] = t["cut_e"][keep]
        t["cut_a"] = t["cut_a"].reshape(-1, B)[keep].reshape(-1)
        t["cut_ptr"] = np.concatenate([t["cut_ptr"][:1], t["cut_ptr"][1:] - B])
        assert e1 - e0 >= B
        return t

    monkeypatch.setattr(pt, "build_block_tree", mutated)
    assert _some_pin_fails([T.test_block_tree_keeps_buses_together_and_factors_each_h_exactly,
                            T.test_block_store_is_the_exact_inverse_and_paper_store_is_algorithm1])


def test_three_phase_fault_with_r_f_as_its_conductance_is_caught(monkeypatch):
    from oracle import emt3
    monkeypatch.setattr(emt3, "fault_conductance", lambda r_f: r_f)
    assert _some_pin_fails([T.test_three_phase_faults_without_mutual_are_single_phase_faults_on_one_copy])


@pytest.mark.parametrize("case", ["none"])
def test_the_pins_pass_without_a_mistake(case):
    # the control: with nothing planted, every pin used above passes
    nw = _tile()
    assert not _some_pin_fails([
        T.test_rc_series_sine_steady_state_bilinear, T.test_rl_sine_steady_state_bilinear,
        T.test_kirchhoff_balance_every_step, T.test_two_bus_golden, T.test_lca_brute_force,
        lambda: T.test_kirchhoff_balance_through_trips_and_overlapping_faults("dense"),
        lambda: T.test_eq5_offdiagonal_blocks_vanish(nw), lambda: T.test_exact_store_equals_dense_inverse(nw),
        lambda: T.test_sherman_morrison_and_woodbury_closed_forms(nw),
        lambda: T.test_algorithm2_to_root_equals_rebuild(nw), T.test_coupled_rl_admittance_closed_form,
        T.test_kl_never_worse_than_growth_and_small_brute_force,
        lambda: T.test_bisection_reaches_brute_force_minimum("ladder", T._graph_ladder(6), 12),
        T.test_three_phase_stepping_without_mutual_is_three_shifted_single_phase_runs,
        T.test_block_tree_keeps_buses_together_and_factors_each_h_exactly,
        T.test_three_phase_faults_without_mutual_are_single_phase_faults_on_one_copy,
        T.test_block_store_is_the_exact_inverse_and_paper_store_is_algorithm1,
        T.test_three_phase_balanced_steady_state_uses_positive_sequence_inductance])
