"""Compile and run the FP64/FP32 issue-rate probe (fp64_peak.cu) and print
the JSON summary that profiles/fp64_peak.txt records."""
import json
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    exe = os.path.join(tempfile.mkdtemp(), "fp64_peak")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    "-DHAVE_M16N8K16", os.path.join(HERE, "fp64_peak.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        d = json.loads(line)
        if "tflops" in d:
            res[d["probe"]] = d["tflops"]
    print(json.dumps({"fp64_tflops": res.get("dfma"), "dmma_fp64_tflops": res.get("dmma_m8n8k4"),
                      "ffma_fp32_tflops": res.get("ffma"), "raw": res}))


if __name__ == "__main__":
    sys.exit(main())
