"""Write workload_terms.json: the percentile-set layer terms of each workload.

The workloads' occurrence retention / limit are the 50th / 99th percentiles
of the generated per-event layer losses, and the aggregate retention / limit
the 10th / 99th percentiles of the trial sums (primary uncertainty,
nearest rank).  They are computed here by the FP64 oracle only
(oracle.calibrate_layer_terms) on the first `sample_trials` trials of the
seeded YET, and stored so that the CUDA path's benchmark and the tests use
the same doubles.  Run:  python tests/golden/make_terms.py

With --serving it writes serving_terms.json instead: the terms of each of the
serving workload's first SERVING_REQUESTS requests (the layer of |J| pool
ELTs and the trial prefix that synth.serving_requests draws), calibrated the
same way on the first min(prefix, SERVING_SAMPLE) trials of its prefix.
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
SERVING_REQUESTS = 10_000
SERVING_SAMPLE = 1000


def _serving_terms(args):
    """Terms of the serving requests [lo, hi) (one worker of a process pool)."""
    lo, hi = args
    spec = synth.WORKLOADS["serving"]
    yet, _, _ = synth.workload("paper-1m", n_trials=SERVING_SAMPLE)
    pool = synth.make_elt_pool(spec["n_elts"], spec["entries"], spec["catalogue"], spec["elt_seed"],
                               recipe=spec["recipe"])
    reqs = synth.serving_requests(spec, hi, spec["request_seed"])[lo:hi]
    out = []
    for ids, t_end in reqs:
        sub = pool.subset([int(j) for j in ids])  # pool ids are the positions 0..n-1
        out.append(list(oracle.calibrate_layer_terms(yet, sub, t_end=min(t_end, SERVING_SAMPLE))))
    return out


def serving() -> None:
    import hashlib
    import multiprocessing as mp

    spec = synth.WORKLOADS["serving"]
    reqs = synth.serving_requests(spec, SERVING_REQUESTS, spec["request_seed"])
    h = hashlib.sha256()
    for ids, t_end in reqs:
        h.update(ids.tobytes())
        h.update(int(t_end).to_bytes(8, "little"))
    os.environ["OMP_NUM_THREADS"] = "1"  # one thread per worker process
    step = 250
    parts = [(lo, min(lo + step, SERVING_REQUESTS)) for lo in range(0, SERVING_REQUESTS, step)]
    with mp.get_context("spawn").Pool(os.cpu_count()) as workers:
        terms = [t for part in workers.map(_serving_terms, parts) for t in part]
    out = {"_source": "percentile-set terms of the serving workload's requests (make_terms.py --serving)",
           "_method": "oracle.calibrate_layer_terms on the first min(prefix, sample_trials) trials of the "
                      "paper-1m YET, primary uncertainty, nearest rank",
           "sample_trials": SERVING_SAMPLE, "requests": SERVING_REQUESTS, "requests_sha256": h.hexdigest(),
           "layer_terms": terms}
    with open(os.path.join(HERE, "serving_terms.json"), "w") as fh:
        json.dump(out, fh, separators=(",", ":"))


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
    if "--serving" in sys.argv:
        serving()
    else:
        main()
