"""Paper-level behaviour (a sanity check of the method, not parity): on the
paper-scale pair (N=2048, N_T=64, the 5 faintest of 33 sources dropped from
epoch 2), augLISI localises the change.  The tiles holding the dropped
sources are exactly its lowest values, while LISI, sensitive to every
intensity change, ranks noise tiles among them (Section 4, the comparison of
the LISI and augLISI maps: augLISI finds source differences with fewer false
positives)."""
import numpy as np

from paper_2501_10653_gb300 import synth

NT = 64
PARAMS = {"C1": 1e-6, "C2": 1e-6, "C": 1e-6, "D": 0.0}


def dropped_tiles():
    xs, ys, _ = synth.paper_pair_dropped()
    T = synth.PAPER_PAIR_N2048["N"] // NT
    return {int(y) // NT * T + int(x) // NT for x, y in zip(xs, ys)}


def check_localisation(lisi, aug):
    tiles = dropped_tiles()
    k = len(tiles)
    assert k == synth.PAPER_PAIR_N2048["n_drop"]  # one dropped source per tile here
    lowest_aug = set(np.argsort(np.asarray(aug).ravel(), kind="stable")[:k].tolist())
    lowest_lisi = set(np.argsort(np.asarray(lisi).ravel(), kind="stable")[:k].tolist())
    assert lowest_aug == tiles
    assert lowest_lisi != tiles


def test_auglisi_localises_dropped_sources_oracle(orc):
    x, y = synth.paper_pair()
    lisi, aug, _ = orc.maps(x, y, NT, PARAMS["C1"], PARAMS["C2"], PARAMS["C"],
                            PARAMS["C1"] / 2, threads=4)
    check_localisation(lisi, aug)
