"""Threshold calibration with the oracle (test infrastructure, run by hand):
``python -m oracle.calibrate``.

The paper leaves S1, S2 and S0 unvalued and reports the rates they give on
its banks; each threshold here is the integer whose rate on random
background proteins (no planted homologs: 200 x 2,000 proteins, seed 1) is
nearest the paper's:

* S1: 0.19 % of the pairs reach the ungapped threshold (the stage-2 pass
  rates of Sections 4.4.3 and 5.4.2, 0.184-0.194 %);
* S2: about 10 % of the stage-3.1 inputs pass (Section 3.3.4: in about 90 %
  of the cases the full gapped extension is not needed);
* S0: 2.5 % of the pairs get through the filter (Section 4.2).  The
  fraction of the unfiltered stage-2 hits the filter keeps is printed beside
  it (Section 4.4.3: 0.165-0.166 % of the pairs pass with the filter against
  0.184-0.186 % without, 89 %).
"""
import numpy as np

import oracle
from paper_0804_3643_gb300 import synth


def background(seed: int = 1):
    rng = np.random.default_rng(seed)
    b1 = synth.random_protein_bank(rng, 200)
    b2 = synth.random_protein_bank(rng, 2000)
    return oracle.make_bank(b1.codes, b1.seq_off), oracle.make_bank(b2.codes, b2.seq_off)


def nearest(rates: dict, target: float) -> int:
    return min(rates, key=lambda t: (abs(rates[t] - target), t))


def main(threads: int = 16) -> dict:
    o1, o2 = background()
    _, pairs = oracle.ungapped(o1, o2, oracle.Params(s1=-10000), threads=threads, return_pairs=True)
    s1_rates = {}
    for s1 in range(30, 47):
        s1_rates[s1] = len(oracle.ungapped(o1, o2, oracle.Params(s1=s1), threads=threads)) / pairs
    s1 = nearest(s1_rates, 0.0019)
    hits = oracle.ungapped(o1, o2, oracle.Params(s1=s1), threads=threads)
    g = oracle.small_gapped(o1, o2, hits, oracle.Params(s1=s1, s2=-30000))
    s2_rates = {s2: float((g["score"] >= s2).mean()) for s2 in range(s1, s1 + 25)}
    s2 = nearest(s2_rates, 0.10)
    s0_rates = {}
    for s0 in range(40, 70):
        _, _, through = oracle.ungapped(o1, o2, oracle.Params(s1=s1, s0=s0), threads=threads, return_pairs=True,
                                        return_filtered=True)
        s0_rates[s0] = through / pairs
    s0 = nearest(s0_rates, 0.025)
    kept = len(oracle.ungapped(o1, o2, oracle.Params(s1=s1, s0=s0), threads=threads)) / len(hits)
    print(f"pairs {pairs}")
    print(f"S1 = {s1}: {100 * s1_rates[s1]:.4f} % of pairs pass stage 2 (target 0.19 %)")
    print(f"S2 = {s2}: {100 * s2_rates[s2]:.2f} % of stage-3.1 inputs pass (target 10 %)")
    print(f"S0 = {s0}: {100 * s0_rates[s0]:.3f} % of pairs through the filter (target 2.5 %), "
          f"{100 * kept:.1f} % of the stage-2 hits kept")
    return {"s1": s1, "s2": s2, "s0": s0}


if __name__ == "__main__":
    main()
