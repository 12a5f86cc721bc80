"""Write the observed images of the benchmark workloads with the FP64 oracle.

For each workload the truth is drawn from the workload's seeded generator
(``inputs.rng_for(workload, 0)``), the noiseless model is the oracle's
(Sec. 2.1.1: supersampled EPL + shear ray shooting, two Sersic lights, k x k
mean, PSF convolution), and seeded noise follows Sec. 2.1.2 / Sec. 3
(Poisson at G t_exp plus Gaussian background), drawn from the same generator
after the truth. Both arms of ``bench.py`` (the CUDA library and the oracle
timed as the reference) and the benchmark's per-result error read these
files, so the data never comes from the CUDA path.

Output: ``<workload>.image.npy`` (float32 [H, W]) and ``<workload>.truth.npy``
(float64 [22]) beside this script. Run from the repository root:
``python tests/golden/bench_inputs/make_bench_images.py``.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2202_07663_gb300 import inputs  # noqa: E402

WORKLOADS = (inputs.MULTISTART, inputs.HMC, inputs.STRESS)


def main():
    for w in WORKLOADS:
        spec = inputs.WORKLOADS[w]["spec"]
        rng = inputs.rng_for(w, 0)
        truth = inputs.draw_truth(rng)
        psf = inputs.make_psf(spec).astype(np.float32)
        model = oracle.simulate(truth, spec.H, spec.W, psf, spec.pixel_scale, spec.k)[0]
        image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
        np.save(os.path.join(HERE, w + ".image.npy"), image)
        np.save(os.path.join(HERE, w + ".truth.npy"), truth.astype(np.float64))
        print(w, image.shape, float(image.sum()))


if __name__ == "__main__":
    main()
