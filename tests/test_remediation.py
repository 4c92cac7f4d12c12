"""Host logic of the Sec. 6.3 trap remediation (paper_2606_30985_gb300.remediation)
against a scripted engine: which runs are retried, with which damping, from
which messages, and what is left in force afterwards."""
import numpy as np
import pytest

from paper_2606_30985_gb300 import PepoError, remediation


class ScriptedEngine:
    """outcome[alpha] = (C, trap_type1); c_drop is reported on the first run."""

    def __init__(self, outcome, alpha=0.5, c_drop=1, n_inst=1):
        self.outcome = outcome
        self.params = (alpha, 1e-5, 100)
        self.c_drop = c_drop
        self.n_inst = n_inst
        self.msgs = np.full(8, 7.0)          # the messages BP starts from
        self.log = []

    def bp_params(self, inst=0):
        return self.params

    def set_bp_params(self, alpha, tol=None, max_sweeps=None, inst=-1):
        self.params = (alpha, tol, max_sweeps)
        self.log.append(("alpha", alpha))

    def get_messages(self, inst=0):
        return self.msgs.copy()

    def set_messages(self, msgs, inst=0):
        self.msgs = np.array(msgs)
        self.log.append(("restore", float(self.msgs[0])))

    def bp_converge(self):
        assert self.msgs[0] == 7.0            # every run starts from the same messages
        self.msgs = self.msgs + 1.0           # BP moves them
        self.log.append(("bp", self.params[0]))
        return [30], [1e-6]

    def correlator(self):
        C, trap = self.outcome[self.params[0]]
        first = sum(1 for e in self.log if e[0] == "bp") == 1
        d = {"C": C, "trap_type1": trap, "c_drop": self.c_drop if first else 0, "bp_sweeps": 40}
        return [C], [d]


def test_clean_layer_is_not_retried():
    eng = ScriptedEngine({0.5: (0.06, 0)})
    C, d, info = remediation.measure(eng)
    assert C == 0.06 and not info["trapped"] and info["retries"] == []
    assert [e for e in eng.log if e[0] == "bp"] == [("bp", 0.5)]


def test_trap_without_a_drop_of_C_is_not_retried():
    eng = ScriptedEngine({0.5: (0.06, 1)}, c_drop=0)
    C, d, info = remediation.measure(eng)
    assert not info["trapped"] and len([e for e in eng.log if e[0] == "bp"]) == 1


def test_confirmed_trap_is_retried_with_the_next_damping():
    eng = ScriptedEngine({0.5: (0.007, 1), 0.8: (0.057, 0), 1.0: (0.058, 0)})
    C, d, info = remediation.measure(eng)
    assert info["trapped"] and info["alpha"] == 0.8 and C == 0.057 and not info["increase_chi"]
    assert [r["alpha"] for r in info["retries"]] == [0.8]
    # the retry starts from the messages of the first run's start, and the
    # damping in force afterwards is the original one
    assert ("restore", 7.0) in eng.log
    assert eng.params[0] == 0.5


def test_undamped_trap_skips_its_own_damping():
    eng = ScriptedEngine({1.0: (0.007, 1), 0.5: (0.066, 0), 0.8: (0.066, 0)}, alpha=1.0)
    C, d, info = remediation.measure(eng)
    assert info["alpha"] == 0.5 and [r["alpha"] for r in info["retries"]] == [0.5]
    assert eng.params[0] == 1.0


def test_every_damping_trapped_asks_for_more_chi_and_restores_the_first_run():
    eng = ScriptedEngine({0.5: (0.007, 1), 0.8: (0.006, 1), 1.0: (0.005, 1)})
    C, d, info = remediation.measure(eng)
    assert info["increase_chi"] and [r["alpha"] for r in info["retries"]] == [0.8, 1.0]
    assert C == 0.007 and eng.params[0] == 0.5
    # measured once more with the original damping, from the same start
    assert eng.log[-3:] == [("alpha", 0.5), ("restore", 7.0), ("bp", 0.5)]


def test_multi_instance_contexts_are_refused():
    with pytest.raises(PepoError):
        remediation.measure(ScriptedEngine({0.5: (0.06, 0)}, n_inst=2))
