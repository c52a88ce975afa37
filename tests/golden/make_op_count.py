"""Writes tests/golden/oracle_op_count.json: the floating-point operations
of one time step per lattice node of the FP64 oracle (its traced build,
oracle/op_count.cpp), for each equation of state.  Calls only oracle/.

  python tests/golden/make_op_count.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

LAWS = {"carnahan_starling": 1, "van_der_waals": 2, "peng_robinson": 3}


def counts():
    return {name: O.op_count(k, 16, 12) for name, k in LAWS.items()}


if __name__ == "__main__":
    doc = {"what": "floating-point operations (add, subtract, multiply, divide, square root) of one oracle time "
                   "step per lattice node, common subexpressions counted once, identities of literals and "
                   "operations on constants not counted (oracle/op_count.cpp)",
           "command": "python tests/golden/make_op_count.py", "lattice": [16, 12], "counts": counts()}
    with open(os.path.join(HERE, "oracle_op_count.json"), "w") as fh:
        json.dump(doc, fh, indent=1)
        fh.write("\n")
    print(json.dumps(doc["counts"]))
