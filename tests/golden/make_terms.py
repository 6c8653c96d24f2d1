"""Write workload_terms.json: the percentile-set layer terms of each workload.

The workloads' occurrence retention / limit are the 50th / 99th percentiles
of the generated per-event layer losses, and the aggregate retention / limit
the 10th / 99th percentiles of the trial sums (primary uncertainty,
nearest rank).  They are computed here by the FP64 oracle only
(oracle.calibrate_layer_terms) on the first `sample_trials` trials of the
seeded YET, and stored so that the CUDA path's benchmark and the tests use
the same doubles.  Run:  python tests/golden/make_terms.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1501_06326_gb300 import synth  # noqa: E402

SAMPLE = {"plain-1k": 1000, "paper-1m": 20000, "stress-1m": 20000}
BATCHED = {"batched-16": 20000}


def main() -> None:
    out = {"_source": __doc__.strip().splitlines()[0], "_method": "oracle.calibrate_layer_terms"}
    for name, n in SAMPLE.items():
        yet, pool, spec = synth.workload(name, n_trials=n)
        terms = oracle.calibrate_layer_terms(yet, pool)
        out[name] = {"sample_trials": n, "layer_terms": list(terms), "elt_ids": pool.elt_ids.tolist()}
        print(name, terms)
    for name, n in BATCHED.items():
        # each layer's terms from its own ELTs, as for a single layer
        yet, pool, spec = synth.workload(name, n_trials=n)
        layers = []
        for ids in synth.workload_layers(spec, pool):
            sub = pool.subset([int(i) for i in ids])  # pool ids are the positions 0..n-1
            terms = oracle.calibrate_layer_terms(yet, sub)
            layers.append({"elt_ids": [int(i) for i in ids], "layer_terms": list(terms)})
        out[name] = {"sample_trials": n, "layers": layers}
        print(name, len(layers), "layers")
    with open(os.path.join(HERE, "workload_terms.json"), "w") as fh:
        json.dump(out, fh, indent=2)


if __name__ == "__main__":
    main()
